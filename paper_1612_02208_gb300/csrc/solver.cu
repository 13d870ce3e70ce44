// libsib: solver context, set-up, V-cycle (Alg. 1), flexible GMRES and the C ABI of sib.h.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <stdexcept>
#include <string>
#include <vector>

#include "sib_internal.h"

using namespace sib;

namespace {

struct SibError : std::runtime_error {
    int code;
    SibError(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define CK(call)                                                                                        \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            throw SibError(SIB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
    } while (0)

constexpr int NBLK = 296;   // fixed block count of the FP64 reductions (2 x 148 ... any fixed value)

template <typename T> struct Prec;
template <> struct Prec<double> { static constexpr int id = 0; };
template <> struct Prec<float> { static constexpr int id = 1; };

}  // namespace

struct LevelBuf {
    void* x = nullptr;
    void* xt = nullptr;
    void* b = nullptr;
    void* r = nullptr;
    void* fib = nullptr;
    void* ibd = nullptr;
    void* w[2] = {nullptr, nullptr};
    // Schur-complement smoother temporaries: 8 velocity-sized, 6 pressure-sized
    void* tv[8] = {};
    void* tp[6] = {};
    void* dinv = nullptr;   // 3 n: SC diagonals
    void* pf = nullptr;     // 7 n: Vanka patch factors
    void* cav = nullptr;    // 5 n: cavity Vanka patch corrections (allocated on first use)
    // Krylov-wrapped smoothing: WRAP_MAXK + 1 Arnoldi vectors, WRAP_MAXK preconditioned ones, a work
    // vector (3 n each) and the step's small FP64 arrays
    void* wV = nullptr;
    void* wZ = nullptr;
    void* ww = nullptr;
    double* wsmall = nullptr;
};

struct Level {
    int N = 0, tx = 0, ty = 0, ntx = 0, nty = 0, ntiles = 0, W = 4;
    double h = 0;
    int* base[2] = {nullptr, nullptr};
    int* binStart[2] = {nullptr, nullptr};
    unsigned char* tileFlag = nullptr;   // 2 * ntiles: raw, dilated
    int* tiles = nullptr;
    int* nTiles = nullptr;
    int hnTiles = 0;
    // slots of the tiles that a marker stencil touches (the raw flag): the rows of the IB operator
    // vanish on the other active tiles (those added by the dilation), whose IB force stays 0
    int* rowSlots = nullptr;
    int* nRowTiles = nullptr;
    int hnRowTiles = 0;
    int spreadWarp = 0;
    LevelBuf p[2];                       // [0] FP64, [1] FP32
    double lamA = 0, lamM = 0;
    // assembled IB operator windows (per active tile), FP64 and FP32
    void* win[2] = {nullptr, nullptr};
    int winSlots = 0;
    int* winOverflow = nullptr;
    int* slotOf = nullptr;               // tile -> slot in the active-tile list, -1 if inactive
    int useWindow = 0;                   // windows valid on this level
    int applyWindow = 0;                 // the solve applies the IB operator through the windows
    // the spreading's walk stored for the marker path (levels that do not apply the windows): row
    // offsets over the faces of the stencil-touched tiles, per-tile counts and offsets, and the
    // entries (marker, weight product in FP64 and FP32)
    int* spLoc = nullptr;
    int* spOff = nullptr;
    int* spTileCnt = nullptr;
    int* spTileOff = nullptr;
    int* spCol = nullptr;
    double* spV64 = nullptr;
    float* spV32 = nullptr;
    size_t spRowsCap = 0, spEntCap = 0;
    bool spReady = false;
    // box RAS smoother: boxes meeting IB windows, their slots, and the owned rows of the subdomain
    // inverses (slot 0 the shared IB-free inverse), FP64 and FP32
    int* rasList = nullptr;
    int* rasSlot = nullptr;
    int* rasCount = nullptr;
    int rasBoxCap = 0;
    void* rasInv[2] = {nullptr, nullptr};
    size_t rasInvCap = 0;                // entries
    int rasNIB = 0;                      // boxes with their own inverse
    float* rasTC = nullptr;              // the shared inverse packed for the tensor-core correction
    size_t rasTCCap = 0;                 // floats
    // a level too small for the boxes: the exact level solve (gauge-fixed pseudo-inverse, FP64)
    bool rasExact = false;
    double* rasPinv = nullptr;
    // 16 x 16 boxes: the full shared inverse (ne x ne, FP64 and FP32) and the IB boxes' Woodbury data
    void* hugeInv[2] = {nullptr, nullptr};
    int* wbOffT = nullptr;               // nIB + 1 offsets into wbT
    int* wbT = nullptr;                  // the IB-touched local dofs of every IB box, ascending
    long long* wbOffW = nullptr;         // nIB offsets into wbW
    double* wbW = nullptr;               // W = (I + E Q)^-1 E per IB box
    double* wbScratch = nullptr;         // (2 mmax + 3 b^2) nIB: y_T, z and y_own of the FP32 levels' IB boxes
    int wbMmax = 0;                      // largest |T|
};

struct sib_ctx {
    int N = 0, n_min = 8, lmax = 0;
    double rho = 0.0, mu = 1.0, dt = 1e-2;
    sib_opts opts{};
    std::string err;
    int64_t launches = 0;
    int smemOptin = 0;           // largest dynamic shared memory of one block
    int64_t bytes = 0;
    double setup_ms = 0.0;
    std::vector<void*> allocs;
    cudaStream_t cap = nullptr;
    void* gjWork = nullptr;              // work arrays of the blocked Gauss-Jordan inversion
    cudaStream_t aux = nullptr;          // set-up work that runs beside the main stream
    cudaEvent_t evFork = nullptr, evJoin = nullptr;
    // the levels' eigenvalue estimates run side by side, one stream (and completion event) per level
    static constexpr int LVS = 16;
    cudaStream_t lvStream[LVS] = {};
    cudaEvent_t lvDone[LVS] = {};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // structure
    int M = 0, E = 0;
    int Mcap = 0, Ecap = 0;
    double* X = nullptr;         // M x 2 interleaved
    double* Xc = nullptr;        // component-major
    int* edges = nullptr;
    double* kappa = nullptr;
    bool structDirty = true, kappaDirty = true, fluidDirty = true, setupDone = false;
    bool haveIB = false;
    // topology
    uint64_t* keys = nullptr;
    int Mpad = 0;
    int* sorted[2] = {nullptr, nullptr};
    uint32_t* mkey[2] = {nullptr, nullptr};
    int* adjStart = nullptr;
    int* adjNbr = nullptr;
    int* adjEid = nullptr;
    int* deg = nullptr;
    double* kap64 = nullptr;
    float* kap32 = nullptr;
    void* U[2] = {nullptr, nullptr};
    void* F[2] = {nullptr, nullptr};
    double* gradTmp = nullptr;   // 8 M: Lam, Y, KY, KL (component-major)
    double* KJ = nullptr;        // 2 x M x 36: per-marker (K J) rows on 6 x 6 patches
    std::vector<Level> L;
    // coarsest
    double* B0 = nullptr;
    double* Aug = nullptr;
    double* Pinv = nullptr;
    int* info = nullptr;
    int* rasInfo = nullptr;      // zero pivot in a box RAS subdomain inverse
    size_t l2Limit = 0;          // the persisting-L2 limit this context set last
    int* piv = nullptr;
    int n0 = 0;
    // FGMRES
    int mcap = 0;
    double* V = nullptr;
    double* Z = nullptr;
    double* rhs = nullptr;
    double* sol = nullptr;
    double* res = nullptr;
    double* part = nullptr;      // NBLK * 128
    double* scal = nullptr;      // 3 * 128 scalars: h, h2, misc
    double* hbuf = nullptr;      // pinned host mirror
    int* herr = nullptr;         // pinned, device-written error word (SIB_DEV_ERR_*), 0 while healthy
    int* flag = nullptr;
    // eigen estimate override
    bool lamOverride = false;
    std::vector<double> lamA_ov, lamM_ov;
    // graphs
    cudaGraphExec_t vg[2] = {nullptr, nullptr};
    void* vgOut[2] = {nullptr, nullptr};
    int64_t vgNodes[2] = {0, 0};
    // device-side FGMRES cycle (conditional graph)
    FgDev* fg = nullptr;
    double* zcur = nullptr;
    cudaGraphExec_t fgExec[2] = {nullptr, nullptr};
    int64_t fgBody[2] = {0, 0}, fgTail[2] = {0, 0};
    bool fgUnavailable = false;
};

namespace {

// the lid-driven cavity instead of the periodic box (option domain)
inline bool cavity(const sib_ctx* c) { return c->opts.domain == SIB_DOMAIN_CAVITY; }

void* dalloc(sib_ctx* c, size_t bytes) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw SibError(SIB_ERR_ALLOC, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    c->allocs.push_back(p);
    c->bytes += (int64_t)bytes;
    return p;
}
void dfree(sib_ctx* c, void* p) {
    if (!p) return;
    for (size_t k = 0; k < c->allocs.size(); ++k)
        if (c->allocs[k] == p) {
            c->allocs.erase(c->allocs.begin() + k);
            break;
        }
    cudaFree(p);
}

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

void kcheck(sib_ctx* c) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw SibError(SIB_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    if (c && c->herr && *(volatile int*)c->herr != 0) {   // a kernel gave up a bounded wait
        const int code = *(volatile int*)c->herr;
        *(volatile int*)c->herr = 0;
        throw SibError(SIB_ERR_CUDA, "device wait ran past its limit (code " + std::to_string(code) +
                                         "): results of the call are invalid");
    }
}

// count one kernel launch (every launcher used on the solve path starts exactly one kernel)
#define KL(c, call)         \
    do {                    \
        call;               \
        ++(c)->launches;    \
    } while (0)

void invalidate_graphs(sib_ctx* c) {
    for (int p = 0; p < 2; ++p) {
        if (c->vg[p]) cudaGraphExecDestroy(c->vg[p]);
        c->vg[p] = nullptr;
        c->vgOut[p] = nullptr;
        if (c->fgExec[p]) cudaGraphExecDestroy(c->fgExec[p]);
        c->fgExec[p] = nullptr;
    }
}

template <typename T>
GridK<T> gridk(sib_ctx* c, int l) {
    Level& lv = c->L[l];
    GridK<T> g;
    g.N = lv.N;
    g.tx = lv.tx;
    g.ty = lv.ty;
    g.ntx = lv.ntx;
    const double h = lv.h;
    g.inv_h = (T)(1.0 / h);
    g.a0 = (T)(c->rho / c->dt + 4.0 * c->mu / (h * h));
    g.c = (T)(c->mu / (h * h));
    g.dt = (T)c->dt;
    g.omega = (T)c->opts.omega;
    const int pi = Prec<T>::id;
    g.fib = (const T*)lv.p[pi].fib;
    g.ibd = (const T*)lv.p[pi].ibd;
    g.tile = c->haveIB ? lv.tileFlag + lv.ntiles : nullptr;
    int lg = 0;
    while ((1 << lg) < lv.tx) ++lg;
    g.lgtx = lg;
    lg = 0;
    while ((1 << lg) < lv.ty) ++lg;
    g.lgty = lg;
    g.dinv = (const T*)lv.p[pi].dinv;
    g.pf = (const T*)lv.p[pi].pf;
    g.err = c->herr;
    return g;
}

template <typename T>
IBK<T> ibk(sib_ctx* c, int l) {
    Level& lv = c->L[l];
    IBK<T> k;
    k.N = lv.N;
    k.W = lv.W;
    k.M = c->M;
    k.shift = 2 * (c->lmax - l);
    const int pi = Prec<T>::id;
    for (int q = 0; q < 2; ++q) {
        k.base[q] = lv.base[q];
        k.wgt[q] = (const T*)lv.p[pi].w[q];
        k.binStart[q] = lv.binStart[q];
        k.sorted[q] = c->sorted[q];
    }
    k.inv_h2 = (T)(1.0 / (lv.h * lv.h));
    return k;
}

template <typename T>
const T* kapp(sib_ctx* c) {
    if constexpr (Prec<T>::id == 0)
        return c->kap64;
    else
        return c->kap32;
}

// dst = x . y (FP64, fixed order); part: NBLK partial sums (default: the context's)
void dot_into(sib_ctx* c, const double* x, const double* y, int64_t n, double* dst, cudaStream_t s,
              double* part = nullptr) {
    if (!part) part = c->part;
    KL(c, launch_dot_partials(x, y, n, part, NBLK, s));
    KL(c, launch_reduce_partials(part, 1, NBLK, dst, s));
}

// f = (1/h^2) S F on the tiles a marker stencil touches: the stored walk where the set-up made it,
// else the cell-binned gather
template <typename T>
void spread_apply(sib_ctx* c, const Level& lv, const IBK<T>& k, const T* F, T* f, cudaStream_t s) {
    if (lv.spReady) {
        const T* val = Prec<T>::id == 0 ? (const T*)(const void*)lv.spV64 : (const T*)(const void*)lv.spV32;
        KL(c, launch_spread_stored<T>(lv.spOff, lv.spCol, val, F, c->M, k.inv_h2, lv.tiles, lv.rowSlots, lv.nRowTiles,
                                      lv.hnRowTiles, lv.N, lv.tx, lv.ty, lv.ntx, f, s));
        return;
    }
    KL(c, launch_spread<T>(k, F, f, lv.tiles, lv.nTiles, lv.hnRowTiles, lv.tx, lv.ty, lv.ntx, lv.spreadWarp, s,
                           lv.rowSlots, lv.nRowTiles));
}

// f = [S K J]^l u (velocity part of x), written into the level's fib (only IB-active tiles)
template <typename T>
void ib_apply(sib_ctx* c, int l, const T* u, cudaStream_t s) {
    if (!c->haveIB) return;
    Level& lv = c->L[l];
    const int pi = Prec<T>::id;
    if (lv.applyWindow) {
        KL(c, launch_ib_window<T>((const T*)lv.win[pi], lv.tiles, lv.rowSlots, lv.nRowTiles, lv.hnRowTiles, lv.N, lv.tx,
                                  lv.ty, lv.ntx, u, (T*)lv.p[pi].fib, s));
        return;
    }
    IBK<T> k = ibk<T>(c, l);
    T* U = (T*)c->U[pi];
    T* F = (T*)c->F[pi];
    KL(c, launch_interp<T>(k, u, U, s));
    KL(c, launch_spring<T>(c->adjStart, c->adjNbr, kapp<T>(c), c->M, U, F, s));
    spread_apply<T>(c, lv, k, F, (T*)lv.p[pi].fib, s);
}

template <typename T>
void apply_operator(sib_ctx* c, int l, const T* x, const T* b, T* r, cudaStream_t s) {
    ib_apply<T>(c, l, x, s);
    if (cavity(c)) {   // r = b - L x, or L x without b; 0 on the wall faces
        if (b)
            KL(c, launch_cavity_residual<T>(gridk<T>(c, l), x, b, r, s));
        else
            KL(c, launch_cavity_apply<T>(gridk<T>(c, l), x, r, s));
        return;
    }
    KL(c, launch_residual<T>(gridk<T>(c, l), x, b, r, s));
}

// ---- Schur-complement smoother (Eq. approx-fact-Stokes-IB) -----------------------------------
struct ChebCoef {
    double theta, delta, sigma;
};
ChebCoef cheb_coef(double lam, double lo, double hi) {
    const double a = lo * lam, b = hi * lam;
    ChebCoef k;
    k.theta = 0.5 * (a + b);
    k.delta = 0.5 * (b - a);
    k.sigma = k.theta / k.delta;
    return k;
}

// z = scale * P_A q and z = scale * P_M q: the point relaxation preconditioning the SC smoother's
// Chebyshev iterations on A_IB and on the Schur complement (option sc_relax): the diagonal inverse,
// or one symmetric red-black Gauss-Seidel sweep from zero (colour passes 0, 1, 1, 0; each pass on
// A_IB first applies the IB operator to the current iterate).
template <typename T>
void precond_A(sib_ctx* c, int l, const T* q, T* z, T scale, cudaStream_t s) {
    GridK<T> g = gridk<T>(c, l);
    if (c->opts.sc_relax != SIB_RELAX_SGS) {
        KL(c, launch_sc_jacobi_A<T>(g, q, z, scale, s));
        return;
    }
    KL(c, launch_sgs_pass<T>(g, false, -1, scale, q, z, s));
    const int order[3] = {1, 1, 0};
    for (int k = 0; k < 3; ++k) {
        ib_apply<T>(c, l, z, s);
        KL(c, launch_sgs_pass<T>(g, false, order[k], scale, q, z, s));
    }
}
template <typename T>
void precond_M(sib_ctx* c, int l, const T* q, T* z, T scale, cudaStream_t s) {
    GridK<T> g = gridk<T>(c, l);
    if (c->opts.sc_relax != SIB_RELAX_SGS) {
        KL(c, launch_jacobi_M<T>(g, q, z, scale, s));
        return;
    }
    KL(c, launch_sgs_pass<T>(g, true, -1, scale, q, z, s));
    const int order[3] = {1, 1, 0};
    for (int k = 0; k < 3; ++k) KL(c, launch_sgs_pass<T>(g, true, order[k], scale, q, z, s));
}

// out = At^{-1} q: cheb_iters Chebyshev iterations on A_IB, preconditioned by P_A, from 0.
// Uses tv[0..3] of the level.
template <typename T>
void cheb_A(sib_ctx* c, int l, const T* q, T* out, cudaStream_t s) {
    Level& lv = c->L[l];
    const int pi = Prec<T>::id;
    const int64_t nv = 2LL * lv.N * lv.N;
    T* rr = (T*)lv.p[pi].tv[0];
    T* t = (T*)lv.p[pi].tv[1];
    T* z = (T*)lv.p[pi].tv[2];
    T* d = (T*)lv.p[pi].tv[3];
    GridK<T> g = gridk<T>(c, l);
    const ChebCoef k = cheb_coef(lv.lamA, c->opts.cheb_lo, c->opts.cheb_hi);
    precond_A<T>(c, l, q, d, (T)(1.0 / k.theta), s);
    KL(c, launch_axpby<T>((T)1, d, (T)0, nullptr, out, nv, s));
    double rho = 1.0 / k.sigma;
    const int iters = c->opts.cheb_iters;
    if (iters > 1) KL(c, launch_axpby<T>((T)1, q, (T)0, nullptr, rr, nv, s));
    for (int it = 1; it < iters; ++it) {
        ib_apply<T>(c, l, d, s);
        KL(c, launch_apply_AIB<T>(g, d, t, s));
        KL(c, launch_axpby<T>((T)1, rr, (T)-1, t, rr, nv, s));
        precond_A<T>(c, l, rr, z, (T)1, s);
        const double rn = 1.0 / (2.0 * k.sigma - rho);
        KL(c, launch_cheb_update<T>(z, d, out, (T)(rn * rho), (T)(2.0 * rn / k.delta), nv, s));
        rho = rn;
    }
}

// out = Mt^{-1} q: Chebyshev iterations on D At^{-1} G preconditioned by P_M (on D diag(A_IB)^{-1} G).
// Uses tv[4..5] and tp[2..5].
template <typename T>
void cheb_M(sib_ctx* c, int l, const T* q, T* out, cudaStream_t s) {
    Level& lv = c->L[l];
    const int pi = Prec<T>::id;
    const int64_t np = (int64_t)lv.N * lv.N;
    T* gq = (T*)lv.p[pi].tv[4];
    T* ya = (T*)lv.p[pi].tv[5];
    T* rr = (T*)lv.p[pi].tp[2];
    T* z = (T*)lv.p[pi].tp[3];
    T* d = (T*)lv.p[pi].tp[4];
    T* md = (T*)lv.p[pi].tp[5];
    GridK<T> g = gridk<T>(c, l);
    const ChebCoef k = cheb_coef(lv.lamM, c->opts.cheb_lo, c->opts.cheb_hi);
    precond_M<T>(c, l, q, d, (T)(1.0 / k.theta), s);
    KL(c, launch_axpby<T>((T)1, d, (T)0, nullptr, out, np, s));
    double rho = 1.0 / k.sigma;
    const int iters = c->opts.cheb_iters;
    if (iters > 1) KL(c, launch_axpby<T>((T)1, q, (T)0, nullptr, rr, np, s));
    for (int it = 1; it < iters; ++it) {
        KL(c, launch_gradient<T>(g, d, gq, s));
        cheb_A<T>(c, l, gq, ya, s);
        KL(c, launch_divergence<T>(g, ya, md, s));
        KL(c, launch_axpby<T>((T)1, rr, (T)-1, md, rr, np, s));
        precond_M<T>(c, l, rr, z, (T)1, s);
        const double rn = 1.0 / (2.0 * k.sigma - rho);
        KL(c, launch_cheb_update<T>(z, d, out, (T)(rn * rho), (T)(2.0 * rn / k.delta), np, s));
        rho = rn;
    }
}

template <typename T>
Cheb2<T> cheb2(double lam, double lo, double hi) {
    const ChebCoef k = cheb_coef(lam, lo, hi);
    const double rho0 = 1.0 / k.sigma, rho1 = 1.0 / (2.0 * k.sigma - rho0);
    Cheb2<T> r;
    r.inv_theta = (T)(1.0 / k.theta);
    r.one_c1 = (T)(1.0 + rho1 * rho0);
    r.c2 = (T)(2.0 * rho1 / k.delta);
    return r;
}

// fused sweep for two Chebyshev iterations per inner solve (6 kernels, plus IB passes on levels
// that use the marker path)
template <typename T>
void sc_sweep_fused(sib_ctx* c, int l, const T* x, const T* b, T* xo, cudaStream_t s, double omega = -1.0) {
    Level& lv = c->L[l];
    const int pi = Prec<T>::id;
    const int64_t nv = 2LL * lv.N * lv.N;
    GridK<T> g = gridk<T>(c, l);
    if (omega >= 0.0) g.omega = (T)omega;
    const Cheb2<T> ka = cheb2<T>(lv.lamA, c->opts.cheb_lo, c->opts.cheb_hi);
    const Cheb2<T> km = cheb2<T>(lv.lamM, c->opts.cheb_lo, c->opts.cheb_hi);
    T* r = (T*)lv.p[pi].r;
    T* y = (T*)lv.p[pi].tv[6];
    T* d = (T*)lv.p[pi].tv[3];
    T* gq = (T*)lv.p[pi].tv[4];
    T* ya = (T*)lv.p[pi].tv[5];
    T* gq2 = (T*)lv.p[pi].tv[0];
    T* dA2 = (T*)lv.p[pi].tv[1];
    T* dA = (T*)lv.p[pi].tv[2];
    T* sv = (T*)lv.p[pi].tp[0];
    T* dp = (T*)lv.p[pi].tp[1];
    T* dM = (T*)lv.p[pi].tp[2];
    if (x) ib_apply<T>(c, l, x, s);   // x == nullptr: zero initial guess, r = b
    KL(c, launch_sc_start<T>(g, ka, x, b, r, d, s));
    ib_apply<T>(c, l, d, s);
    KL(c, launch_sc_chebA<T>(g, ka, r, d, y, s));
    KL(c, launch_sc_mstart<T>(g, ka, km, r + nv, y, sv, dM, gq, dA, s));
    ib_apply<T>(c, l, dA, s);
    KL(c, launch_sc_chebA<T>(g, ka, gq, dA, ya, s));
    KL(c, launch_sc_mfinish<T>(g, ka, km, sv, dM, ya, dp, gq2, dA2, s));
    ib_apply<T>(c, l, dA2, s);
    KL(c, launch_sc_finish<T>(g, ka, x, y, gq2, dA2, dp, xo, s));
}

// the fused SC sweep covers two Chebyshev iterations with Jacobi relaxation
bool sc_fused(const sib_ctx* c) { return c->opts.cheb_iters == 2 && c->opts.sc_relax == SIB_RELAX_JACOBI; }

// xo = x + omega * Lt^{-1} (b - L x)  (x == nullptr: zero initial guess; omega < 0: the option's)
template <typename T>
void sc_sweep(sib_ctx* c, int l, const T* x, const T* b, T* xo, cudaStream_t s, double omega = -1.0) {
    if (sc_fused(c)) {
        sc_sweep_fused<T>(c, l, x, b, xo, s, omega);
        return;
    }
    Level& lv = c->L[l];
    const int pi = Prec<T>::id;
    const int64_t np = (int64_t)lv.N * lv.N, nv = 2 * np;
    T* r = (T*)lv.p[pi].r;
    T* y = (T*)lv.p[pi].tv[6];
    T* yy = (T*)lv.p[pi].tv[7];
    T* sv = (T*)lv.p[pi].tp[0];
    T* dp = (T*)lv.p[pi].tp[1];
    GridK<T> g = gridk<T>(c, l);
    if (x)
        apply_operator<T>(c, l, x, b, r, s);
    else
        KL(c, launch_axpby<T>((T)1, b, (T)0, nullptr, r, nv + np, s));
    cheb_A<T>(c, l, r, y, s);                                        // y = At^{-1} r_u
    KL(c, launch_divergence<T>(g, y, sv, s));                        // s = r_p + D y
    KL(c, launch_axpby<T>((T)1, r + nv, (T)1, sv, sv, np, s));
    cheb_M<T>(c, l, sv, dp, s);                                      // dp = Mt^{-1} s
    T* gq = (T*)lv.p[pi].tv[4];
    KL(c, launch_gradient<T>(g, dp, gq, s));                         // yy = At^{-1} G dp
    cheb_A<T>(c, l, gq, yy, s);
    const T om = (T)(omega >= 0.0 ? omega : c->opts.omega);
    KL(c, launch_axpby<T>((T)1, y, (T)-1, yy, y, nv, s));            // du = y - yy
    if (x) {
        KL(c, launch_axpby<T>((T)1, x, om, y, xo, nv, s));           // xo_u = x_u + omega du
        KL(c, launch_axpby<T>((T)1, x + nv, om, dp, xo + nv, np, s));   // xo_p = x_p + omega dp
    } else {
        KL(c, launch_axpby<T>(om, y, (T)0, nullptr, xo, nv, s));
        KL(c, launch_axpby<T>(om, dp, (T)0, nullptr, xo + nv, np, s));
    }
}

// the packed shared inverse when the IB-free boxes of an FP32 level take the tensor-core correction
template <typename T>
const float* ras_tc_pack_for(const sib_ctx* c, const Level& lv) {
    return (Prec<T>::id == 1 && c->opts.ras_tc) ? lv.rasTC : nullptr;
}

// one RAS correction on level l: xo = x + omega Rt^T L_k^{-1} r (x == nullptr: zero initial guess; x and xo
// are distinct buffers)
template <typename T>
void ras_apply(sib_ctx* c, int l, const T* r, const T* x, T* xo, double omega, cudaStream_t s) {
    Level& lv = c->L[l];
    const int pi = Prec<T>::id;
    const int b = c->opts.box, o = c->opts.box_overlap;
    if (lv.rasExact) {   // a level too small for the boxes: the exact level solve
        KL(c, launch_dense_correct<T>(lv.rasPinv, 3 * lv.N * lv.N, r, x, (T)omega, xo, s));
        return;
    }
    if (ras_huge(b)) {   // 16 x 16 boxes: the shared correction of every box, then the IB boxes' update
        bool done = false;
        if (Prec<T>::id == 1 && c->opts.ras_tc && (lv.N / b) * (lv.N / b) >= RAS_TC_MIN_BOXES) {
            done = launch_ras_apply_tc_groups(lv.N, b, o, lv.rasTC, 3 * b * b / RAS_TC_GROUP, (float)omega,
                                              (const float*)r, (const float*)x, (float*)xo, c->herr, s);
            if (done) ++c->launches;
        }
        if (!done) KL(c, launch_ras_huge_apply<T>(lv.N, b, o, (const T*)lv.hugeInv[pi], (T)omega, r, x, xo, s));
        if (lv.rasNIB > 0) {
            const RasIB ib{lv.slotOf, (const double*)lv.win[0], lv.tx, lv.ty, lv.ntx};
            const double h = lv.h, a0 = c->rho / c->dt + 4.0 * c->mu / (h * h), cc = c->mu / (h * h);
            KL(c, launch_ras_wb_apply<T>(lv.N, b, o, ib, a0, cc, 1.0 / h, c->dt, lv.rasList, lv.rasNIB, lv.wbOffT,
                                         lv.wbT, lv.wbOffW, lv.wbW, (const double*)lv.hugeInv[0], lv.wbMmax,
                                         (T)omega, r, xo, s, lv.wbScratch, x));
            if (Prec<T>::id == 1) c->launches += 2;   // the FP32 form is three launches
        }
        return;
    }
    const float* tc = ras_tc_pack_for<T>(c, lv);
    KL(c, launch_ras_apply<T>(lv.N, c->opts.box, c->opts.box_overlap, lv.rasSlot, lv.rasList, lv.rasNIB,
                              (const T*)lv.rasInv[pi], (T)omega, r, x, xo, s, tc, c->herr));
    if (lv.rasNIB > 0) ++c->launches;
}

// one smoothing sweep xo <- smooth(x, b)
template <typename T>
void sweep(sib_ctx* c, int l, const T* x, const T* b, T* xo, cudaStream_t s) {
    if (cavity(c)) {   // the cavity's Vanka sweep: residual, patch solves with the wall rules, update
        LevelBuf& lb = c->L[l].p[Prec<T>::id];
        ib_apply<T>(c, l, x, s);
        launch_cavity_vanka<T>(gridk<T>(c, l), x, b, (T*)lb.r, (T*)lb.cav, xo, (T)c->opts.omega, s);
        c->launches += 3;
    } else if (c->opts.smoother == SIB_SMOOTHER_SC) {
        sc_sweep<T>(c, l, x, b, xo, s);
    } else if (c->opts.smoother == SIB_SMOOTHER_RAS) {   // r = b - L x, then the box corrections
        T* r = (T*)c->L[l].p[Prec<T>::id].r;
        ib_apply<T>(c, l, x, s);
        KL(c, launch_residual<T>(gridk<T>(c, l), x, b, r, s));
        ras_apply<T>(c, l, r, x, xo, c->opts.omega, s);
    } else {
        ib_apply<T>(c, l, x, s);
        KL(c, launch_vanka<T>(gridk<T>(c, l), x, b, xo, s));
    }
}

// Levels 1 and 0 fit one thread block's shared memory (kernels_small.cu): level 1 of at most
// 16 x 16 cells, its IB operator (if any) applied through windows, the fused SC sweep.
template <typename T>
size_t small_smem(const sib_ctx* c) {
    const Level& lv = c->L[1];
    const int nT = c->haveIB ? lv.hnTiles : 0;
    return vcycle_small_smem<T>(lv.N, c->n0, nT, lv.tx * lv.ty, lv.ntiles);
}
template <typename T>
bool small_ok(const sib_ctx* c) {
    if (!c->opts.fuse_small || c->lmax < 1 || cavity(c)) return false;
    const Level& lv = c->L[1];
    if (lv.N > 16) return false;
    if (c->opts.smoother == SIB_SMOOTHER_SC && !sc_fused(c)) return false;
    if (c->opts.smoother == SIB_SMOOTHER_RAS) return false;
    if (c->haveIB && lv.hnTiles > 0 && !lv.applyWindow) return false;
    const size_t smem = small_smem<T>(c);
    if (smem > (size_t)c->smemOptin) return false;
    // the coarse-solve helpers hold the pseudo-inverse's rows in the same shared-memory size
    if (sizeof(double) * ((size_t)(c->n0 + 6) / 7 + 1) * c->n0 > smem) return false;
    return vcycle_small_cluster<T>(smem) > 0;
}
template <typename T>
T* vcycle_small(sib_ctx* c, cudaStream_t s) {
    Level& lv = c->L[1];
    const int pi = Prec<T>::id;
    SmallArgs<T> a{};
    a.g = gridk<T>(c, 1);
    if (c->opts.smoother == SIB_SMOOTHER_SC) {
        a.ka = cheb2<T>(lv.lamA, c->opts.cheb_lo, c->opts.cheb_hi);
        a.km = cheb2<T>(lv.lamM, c->opts.cheb_lo, c->opts.cheb_hi);
    }
    a.b = (const T*)lv.p[pi].b;
    a.out = (T*)lv.p[pi].x;
    a.win = (const T*)lv.win[pi];
    a.tiles = lv.tiles;
    a.nTiles = c->haveIB ? lv.hnTiles : 0;
    a.ntiles = lv.ntiles;
    a.smoother = c->opts.smoother;
    a.nu1 = c->opts.nu1;
    a.nu2 = c->opts.nu2;
    a.n0 = c->n0;
    a.Pinv = c->Pinv;
    CK(launch_vcycle_small<T>(a, small_smem<T>(c), s));
    ++c->launches;
    return (T*)lv.p[pi].x;
}

// Krylov-wrapped smoothing step (Sec. 3.3): xo = x + e, e from k iterations of flexible GMRES on
// L e = b - L x (CGS2), each preconditioned by one undamped sweep of the basic smoother from zero;
// x == nullptr: zero start.  The Hessenberg least-squares problem is solved on the device.
template <typename T>
void wrapped_smooth(sib_ctx* c, int l, const T* x, const T* b, T* xo, int k, cudaStream_t s) {
    Level& lv = c->L[l];
    const int pi = Prec<T>::id;
    LevelBuf& lb = lv.p[pi];
    const int64_t n3 = 3LL * lv.N * lv.N;
    const int K1 = WRAP_MAXK + 1;
    T* V = (T*)lb.wV;
    T* Z = (T*)lb.wZ;
    T* w = (T*)lb.ww;
    double* hA = lb.wsmall;
    double* hB = hA + K1 * WRAP_MAXK;
    double* nr = hB + K1 * WRAP_MAXK;
    double* beta2 = nr + WRAP_MAXK;
    double* y = beta2 + 1;
    double* part = y + WRAP_MAXK;
    // small levels: one block forms every inner product and norm, without a reduce kernel
    const bool one = n3 <= WRAP_ONE_MAX;
    auto dots = [&](const T* Vs, int cnt, const T* v, double* out) {
        if (one) {
            KL(c, launch_wdots<T>(Vs, n3, cnt, v, n3, out, s));
            return;
        }
        const int nb = launch_wdots<T>(Vs, n3, cnt, v, n3, part, s);
        KL(c, launch_wreduce(part, cnt, nb, out, s));
        ++c->launches;
    };
    const T* r0 = b;
    if (x) {
        apply_operator<T>(c, l, x, b, w, s);   // r = b - L x
        r0 = w;
    }
    if (one) {
        KL(c, launch_wnorm_one<T>(r0, n3, beta2, V, s));
    } else {
        dots(r0, 1, r0, beta2);
        KL(c, launch_wscale<T>(r0, beta2, V, n3, s));
    }
    GridK<T> g = gridk<T>(c, l);
    g.omega = T(1);   // the basic smoother undamped
    for (int j = 0; j < k; ++j) {
        T* Vj = V + (size_t)j * n3;
        T* Zj = Z + (size_t)j * n3;
        if (c->opts.smoother == SIB_SMOOTHER_SC)
            sc_sweep<T>(c, l, nullptr, Vj, Zj, s, 1.0);
        else if (c->opts.smoother == SIB_SMOOTHER_RAS)
            ras_apply<T>(c, l, Vj, nullptr, Zj, 1.0, s);
        else
            KL(c, launch_vanka_zero<T>(g, Vj, Zj, s));
        ib_apply<T>(c, l, Zj, s);
        KL(c, launch_residual<T>(gridk<T>(c, l), Zj, nullptr, w, s));   // w = L z_j
        // CGS2: h = V^T w; w -= V h and h' = V^T w in one pass; w -= V h' and |w|^2 in one pass
        dots(V, j + 1, w, hA + j * K1);
        if (one) {
            KL(c, launch_wgs<T>(V, n3, j + 1, hA + j * K1, w, w, n3, 1, hB + j * K1, s));
            KL(c, launch_wgs2_one<T>(V, n3, j + 1, hB + j * K1, w, n3, nr + j,
                                     j + 1 < k ? V + (size_t)(j + 1) * n3 : nullptr, j + 1 < k ? 0 : k, hA, hB, nr,
                                     beta2, y, s));
            continue;
        }
        int nb = launch_wgs<T>(V, n3, j + 1, hA + j * K1, w, w, n3, 1, part, s);
        KL(c, launch_wreduce(part, j + 1, nb, hB + j * K1, s));
        nb = launch_wgs<T>(V, n3, j + 1, hB + j * K1, w, w, n3, 2, part, s);
        if (j + 1 < k)
            KL(c, launch_wreduce(part, 1, nb, nr + j, s));
        else   // the stage's last norm and its least-squares solve
            KL(c, launch_wreduce_lsq(part, nb, nr + j, hA, hB, nr, beta2, k, y, s));
        c->launches += 2;
        if (j + 1 < k) KL(c, launch_wscale<T>(w, nr + j, V + (size_t)(j + 1) * n3, n3, s));
    }
    KL(c, launch_wmaxpy<T>(Z, n3, k, y, 1.0, x, xo, n3, s));
}

// Alg. 1 on level l with right-hand side in the level's b; returns the buffer holding w.
template <typename T>
T* vcycle_level(sib_ctx* c, int l, cudaStream_t s) {
    Level& lv = c->L[l];
    const int pi = Prec<T>::id;
    if (l == 1 && !c->opts.smooth_krylov && small_ok<T>(c)) return vcycle_small<T>(c, s);
    if (l == 0) {
        KL(c, launch_coarse_apply<T>(c->Pinv, c->n0, (const T*)lv.p[pi].b, (T*)lv.p[pi].x, s));
        return (T*)lv.p[pi].x;
    }
    if (cavity(c)) {   // the lid-driven cavity: wall-rule sweeps and the walled transfers
        T* x = (T*)lv.p[pi].x;
        T* xt = (T*)lv.p[pi].xt;
        const T* b = (const T*)lv.p[pi].b;
        CK(cudaMemsetAsync(x, 0, sizeof(T) * 3 * (size_t)lv.N * lv.N, s));
        for (int k = 0; k < c->opts.nu1; ++k) {
            sweep<T>(c, l, x, b, xt, s);
            std::swap(x, xt);
        }
        T* r = (T*)lv.p[pi].r;
        apply_operator<T>(c, l, x, b, r, s);
        KL(c, launch_cavity_restrict<T>(c->L[l - 1].N, r, (T*)c->L[l - 1].p[pi].b, s));
        T* ec = vcycle_level<T>(c, l - 1, s);
        KL(c, launch_cavity_prolong_add<T>(c->L[l - 1].N, ec, x, s));
        for (int k = 0; k < c->opts.nu2; ++k) {
            sweep<T>(c, l, x, b, xt, s);
            std::swap(x, xt);
        }
        return x;
    }
    if (c->opts.smooth_krylov) {   // each smoothing stage: FGMRES(nu) preconditioned by the basic sweep
        T* x = (T*)lv.p[pi].x;
        T* xt = (T*)lv.p[pi].xt;
        const T* b = (const T*)lv.p[pi].b;
        if (c->opts.nu1 > 0)
            wrapped_smooth<T>(c, l, (const T*)nullptr, b, x, c->opts.nu1, s);
        else
            CK(cudaMemsetAsync(x, 0, sizeof(T) * 3 * (size_t)lv.N * lv.N, s));
        ib_apply<T>(c, l, x, s);
        KL(c, launch_residual_restrict<T>(gridk<T>(c, l), x, b, (T*)c->L[l - 1].p[pi].b, s));
        T* ec = vcycle_level<T>(c, l - 1, s);
        KL(c, launch_prolong_add<T>(c->L[l - 1].N, ec, x, s));
        if (c->opts.nu2 > 0) {
            wrapped_smooth<T>(c, l, (const T*)x, b, xt, c->opts.nu2, s);
            std::swap(x, xt);
        }
        return x;
    }
    const int64_t n3 = 3LL * lv.N * lv.N;
    T* x = (T*)lv.p[pi].x;
    T* xt = (T*)lv.p[pi].xt;
    const T* b = (const T*)lv.p[pi].b;
    int k0 = 0;
    if (c->opts.smoother == SIB_SMOOTHER_VANKA && c->opts.nu1 > 0) {
        KL(c, launch_vanka_zero<T>(gridk<T>(c, l), b, xt, s));   // first sweep from w = 0
        std::swap(x, xt);
        k0 = 1;
    } else if (c->opts.smoother == SIB_SMOOTHER_SC && c->opts.nu1 > 0) {
        sc_sweep<T>(c, l, nullptr, b, xt, s);   // first sweep from w = 0: residual = b
        std::swap(x, xt);
        k0 = 1;
    } else if (c->opts.smoother == SIB_SMOOTHER_RAS && c->opts.nu1 > 0) {
        ras_apply<T>(c, l, b, nullptr, xt, c->opts.omega, s);   // first sweep from w = 0: residual = b
        std::swap(x, xt);
        k0 = 1;
    } else {
        CK(cudaMemsetAsync(x, 0, sizeof(T) * n3, s));
    }
    for (int k = k0; k < c->opts.nu1; ++k) {
        sweep<T>(c, l, x, b, xt, s);
        std::swap(x, xt);
    }
    ib_apply<T>(c, l, x, s);
    KL(c, launch_residual_restrict<T>(gridk<T>(c, l), x, b, (T*)c->L[l - 1].p[pi].b, s));
    T* ec = vcycle_level<T>(c, l - 1, s);
    KL(c, launch_prolong_add<T>(c->L[l - 1].N, ec, x, s));
    for (int k = 0; k < c->opts.nu2; ++k) {
        sweep<T>(c, l, x, b, xt, s);
        std::swap(x, xt);
    }
    return x;
}

// The capture stream's L2 access policy, which the captured kernels keep: the finest level's FP32 IB
// windows, read by several passes of every sweep, persist in L2 (option l2_persist), within this
// process's persisting-L2 limit (set to their size, at most the device's maximum).
void apply_l2_policy(sib_ctx* c) {
    cudaStreamAttrValue v{};
    size_t limit = 0;
    const Level& lv = c->L[c->lmax];
    const size_t bytes = c->haveIB && lv.applyWindow && lv.win[1]
                             ? sizeof(float) * (size_t)lv.hnTiles * 2 * WIN_SIZE * lv.tx * lv.ty
                             : 0;
    if (c->opts.l2_persist && bytes > 0) {
        int dev = 0, maxPersist = 0, maxWin = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&maxPersist, cudaDevAttrMaxPersistingL2CacheSize, dev));
        CK(cudaDeviceGetAttribute(&maxWin, cudaDevAttrMaxAccessPolicyWindowSize, dev));
        const size_t win = std::min(bytes, (size_t)maxWin);
        const size_t persist = std::min(win, (size_t)maxPersist);
        if (persist > 0) {
            limit = persist;
            v.accessPolicyWindow.base_ptr = lv.win[1];
            v.accessPolicyWindow.num_bytes = win;
            v.accessPolicyWindow.hitRatio = (float)((double)persist / (double)win);
            v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
            v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
        }
    }
    if (limit != c->l2Limit) {   // the limit reconfigures the L2: set (or release) it only when it changes
        CK(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, limit));
        c->l2Limit = limit;
    }
    CK(cudaStreamSetAttribute(c->cap, cudaStreamAttributeAccessPolicyWindow, &v));
}

// Run one V-cycle on the finest level's b; returns the output buffer.
template <typename T>
T* vcycle(sib_ctx* c, cudaStream_t s) {
    const int pi = Prec<T>::id;
    if (!c->opts.use_graphs) return vcycle_level<T>(c, c->lmax, s);
    if (!c->vg[pi]) {
        const int64_t before = c->launches;
        cudaGraph_t graph;
        apply_l2_policy(c);
        CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        T* out = nullptr;
        try {
            out = vcycle_level<T>(c, c->lmax, c->cap);
        } catch (...) {
            cudaStreamEndCapture(c->cap, &graph);
            throw;
        }
        CK(cudaStreamEndCapture(c->cap, &graph));
        CK(cudaGraphInstantiate(&c->vg[pi], graph, 0));
        cudaGraphDestroy(graph);
        c->vgOut[pi] = out;
        c->vgNodes[pi] = c->launches - before;
        c->launches = before;
    }
    CK(cudaGraphLaunch(c->vg[pi], s));
    c->launches += c->vgNodes[pi];
    return (T*)c->vgOut[pi];
}

int64_t n3f(sib_ctx* c) { return 3LL * c->N * c->N; }

// ---- set-up -----------------------------------------------------------------------------------
void alloc_level_bufs(sib_ctx* c) {
    for (int l = 0; l <= c->lmax; ++l) {
        Level& lv = c->L[l];
        const size_t n = (size_t)lv.N * lv.N;
        for (int pi = 0; pi < 2; ++pi) {
            const size_t e = pi == 0 ? 8 : 4;
            LevelBuf& b = lv.p[pi];
            b.x = dalloc(c, e * 3 * n);
            b.xt = dalloc(c, e * 3 * n);
            b.b = dalloc(c, e * 3 * n);
            b.r = dalloc(c, e * 3 * n);
            b.fib = dalloc(c, e * 2 * n);
            b.ibd = dalloc(c, e * 4 * n);
            b.pf = dalloc(c, e * 7 * n);
        }
        lv.tileFlag = (unsigned char*)dalloc(c, 2 * (size_t)lv.ntiles);
        lv.tiles = (int*)dalloc(c, sizeof(int) * (size_t)lv.ntiles);
        lv.slotOf = (int*)dalloc(c, sizeof(int) * (size_t)lv.ntiles);
        lv.nTiles = (int*)dalloc(c, sizeof(int));
        lv.rowSlots = (int*)dalloc(c, sizeof(int) * (size_t)lv.ntiles);
        lv.nRowTiles = (int*)dalloc(c, sizeof(int));
        lv.binStart[0] = (int*)dalloc(c, sizeof(int) * (n + 1));
        lv.binStart[1] = (int*)dalloc(c, sizeof(int) * (n + 1));
    }
}

// Krylov-wrapped smoothing buffers of every level >= 1, both precisions (once; WRAP_MAXK-sized)
void alloc_wrap_bufs(sib_ctx* c) {
    for (int l = 1; l <= c->lmax; ++l) {
        Level& lv = c->L[l];
        const size_t n3 = 3 * (size_t)lv.N * lv.N;
        for (int pi = 0; pi < 2; ++pi) {
            const size_t e = pi == 0 ? 8 : 4;
            LevelBuf& b = lv.p[pi];
            if (b.wV) continue;
            b.wV = dalloc(c, e * n3 * (WRAP_MAXK + 1));
            b.wZ = dalloc(c, e * n3 * WRAP_MAXK);
            b.ww = dalloc(c, e * n3);
            const size_t small = 2 * (size_t)(WRAP_MAXK + 1) * WRAP_MAXK + WRAP_MAXK + 1 + WRAP_MAXK +
                                 (size_t)(WRAP_MAXK + 1) * WRAP_BLK;
            b.wsmall = (double*)dalloc(c, sizeof(double) * small);
        }
    }
}

void alloc_sc_bufs(sib_ctx* c) {
    for (int l = 1; l <= c->lmax; ++l) {
        Level& lv = c->L[l];
        const size_t n = (size_t)lv.N * lv.N;
        for (int pi = 0; pi < 2; ++pi) {
            const size_t e = pi == 0 ? 8 : 4;
            LevelBuf& b = lv.p[pi];
            if (b.tv[0]) continue;
            for (int k = 0; k < 8; ++k) b.tv[k] = dalloc(c, e * 2 * n);
            for (int k = 0; k < 6; ++k) b.tp[k] = dalloc(c, e * n);
            b.dinv = dalloc(c, e * 3 * n);
        }
    }
}

void alloc_markers(sib_ctx* c) {
    if (c->M <= c->Mcap && c->E <= c->Ecap && c->X) return;
    for (int l = 0; l <= c->lmax; ++l) {
        Level& lv = c->L[l];
        for (int q = 0; q < 2; ++q) {
            dfree(c, lv.base[q]);
            dfree(c, lv.p[0].w[q]);
            dfree(c, lv.p[1].w[q]);
        }
    }
    for (void* p : {(void*)c->X, (void*)c->Xc, (void*)c->edges, (void*)c->kappa, (void*)c->keys, (void*)c->sorted[0],
                    (void*)c->sorted[1], (void*)c->mkey[0], (void*)c->mkey[1], (void*)c->adjStart, (void*)c->adjNbr,
                    (void*)c->adjEid, (void*)c->deg, (void*)c->kap64, (void*)c->kap32, c->U[0], c->U[1], c->F[0],
                    c->F[1], (void*)c->gradTmp, (void*)c->KJ})
        dfree(c, p);
    const int Mc = c->M > c->Mcap ? c->M : (c->Mcap > 0 ? c->Mcap : 1);
    const int Ec = c->E > c->Ecap ? c->E : (c->Ecap > 0 ? c->Ecap : 1);
    c->Mcap = Mc;
    c->Ecap = Ec;
    int Mpad = 1;
    while (Mpad < Mc) Mpad <<= 1;
    c->X = (double*)dalloc(c, sizeof(double) * 2 * Mc);
    c->Xc = (double*)dalloc(c, sizeof(double) * 2 * Mc);
    c->edges = (int*)dalloc(c, sizeof(int) * 2 * Ec);
    c->kappa = (double*)dalloc(c, sizeof(double) * Ec);
    c->keys = (uint64_t*)dalloc(c, sizeof(uint64_t) * Mpad);
    for (int q = 0; q < 2; ++q) {
        c->sorted[q] = (int*)dalloc(c, sizeof(int) * Mc);
        c->mkey[q] = (uint32_t*)dalloc(c, sizeof(uint32_t) * Mc);
    }
    c->adjStart = (int*)dalloc(c, sizeof(int) * (Mc + 1));
    c->adjNbr = (int*)dalloc(c, sizeof(int) * 2 * Ec);
    c->adjEid = (int*)dalloc(c, sizeof(int) * 2 * Ec);
    c->deg = (int*)dalloc(c, sizeof(int) * Mc);
    c->kap64 = (double*)dalloc(c, sizeof(double) * 2 * Ec);
    c->kap32 = (float*)dalloc(c, sizeof(float) * 2 * Ec);
    c->U[0] = dalloc(c, sizeof(double) * 2 * Mc);
    c->F[0] = dalloc(c, sizeof(double) * 2 * Mc);
    c->U[1] = dalloc(c, sizeof(float) * 2 * Mc);
    c->F[1] = dalloc(c, sizeof(float) * 2 * Mc);
    c->gradTmp = (double*)dalloc(c, sizeof(double) * 8 * Mc);
    c->KJ = (double*)dalloc(c, sizeof(double) * 2 * 36 * (size_t)Mc);
    for (int l = 0; l <= c->lmax; ++l) {
        Level& lv = c->L[l];
        for (int q = 0; q < 2; ++q) {
            lv.base[q] = (int*)dalloc(c, sizeof(int) * Mc);
            lv.p[0].w[q] = dalloc(c, sizeof(double) * 8 * Mc);
            lv.p[1].w[q] = dalloc(c, sizeof(float) * 8 * Mc);
        }
    }
}

void alloc_krylov(sib_ctx* c) {
    const int m = c->opts.restart < c->opts.max_it ? c->opts.restart : c->opts.max_it;
    if (m <= c->mcap && c->V) return;
    dfree(c, c->V);
    dfree(c, c->Z);
    const size_t n = (size_t)n3f(c);
    c->V = (double*)dalloc(c, sizeof(double) * n * (m + 1));
    c->Z = (double*)dalloc(c, sizeof(double) * n * m);
    c->mcap = m;
}

// Power iterations for lambda_max of DA^{-1} A_IB and of DM^{-1} D At^{-1} G on level l (FP64),
// from the normalised hash start vector, without renormalising between steps (the growth over the
// steps stays far inside FP64's range): ||A v||^2 of the last step lands in scal[slot] and ||v||^2 in
// scal[slot + 40], so that lambda = (||A v|| / ||v||), the normalised iteration's estimate (setup reads
// all levels back with one synchronisation per operator).  A level's chain touches only that level's
// buffers, its slots and its own NBLK partial sums (part).
void power_A_enqueue(sib_ctx* c, int l, int slot, double* part, cudaStream_t s) {
    Level& lv = c->L[l];
    const int64_t nv = 2LL * lv.N * lv.N;
    double* v = (double*)lv.p[0].tv[6];
    double* w = (double*)lv.p[0].tv[7];
    GridK<double> g = gridk<double>(c, l);
    KL(c, launch_hash_vector(v, nv, s));
    dot_into(c, v, v, nv, c->scal + slot, s, part);
    KL(c, launch_scale(v, c->scal, slot, nv, s));
    for (int it = 0; it < c->opts.power_iters; ++it) {
        ib_apply<double>(c, l, v, s);
        if (c->opts.sc_relax == SIB_RELAX_SGS) {   // w = P_A A_IB v
            double* t = (double*)lv.p[0].tv[0];
            KL(c, launch_apply_AIB<double>(g, v, t, s));
            precond_A<double>(c, l, t, w, 1.0, s);
        } else {
            KL(c, launch_power_A<double>(g, v, w, s));
        }
        if (it + 1 < c->opts.power_iters) std::swap(v, w);
    }
    dot_into(c, w, w, nv, c->scal + slot, s, part);
    dot_into(c, v, v, nv, c->scal + slot + 40, s, part);
}
void power_M_enqueue(sib_ctx* c, int l, int slot, double* part, cudaStream_t s) {
    Level& lv = c->L[l];
    const int64_t np = (int64_t)lv.N * lv.N;
    double* v = (double*)lv.p[0].tp[0];
    double* w = (double*)lv.p[0].tp[1];
    double* md = (double*)lv.p[0].tp[5];
    double* gq = (double*)lv.p[0].tv[4];
    double* ya = (double*)lv.p[0].tv[5];
    double* dA = (double*)lv.p[0].tv[2];
    GridK<double> g = gridk<double>(c, l);
    const Cheb2<double> ka = cheb2<double>(lv.lamA, c->opts.cheb_lo, c->opts.cheb_hi);
    KL(c, launch_hash_vector(v, np, s));
    dot_into(c, v, v, np, c->scal + slot, s, part);
    KL(c, launch_scale(v, c->scal, slot, np, s));
    for (int it = 0; it < c->opts.power_iters; ++it) {
        if (sc_fused(c)) {
            KL(c, launch_power_Mstart<double>(g, ka, v, gq, dA, s));
            ib_apply<double>(c, l, dA, s);
            KL(c, launch_sc_chebA<double>(g, ka, gq, dA, ya, s));
            KL(c, launch_power_Mfinish<double>(g, ya, w, s));
        } else {
            KL(c, launch_gradient<double>(g, v, gq, s));
            cheb_A<double>(c, l, gq, ya, s);
            KL(c, launch_divergence<double>(g, ya, md, s));
            precond_M<double>(c, l, md, w, 1.0, s);
        }
        if (it + 1 < c->opts.power_iters) std::swap(v, w);
    }
    dot_into(c, w, w, np, c->scal + slot, s, part);
    dot_into(c, v, v, np, c->scal + slot + 40, s, part);
}

// Box RAS set-up on levels 1..lmax (Sec. 3.3, Alg. 2 with boxes): classify the boxes by whether
// their subdomain meets an IB window, then assemble and invert the shared IB-free subdomain operator
// and one per IB box (FP64), keeping the owned rows of each inverse.  Wide subdomains are eliminated
// in a temporary global workspace, at most RAS_WORK_BYTES of matrices per launch.
constexpr size_t RAS_WORK_BYTES = size_t(1) << 31;
// The RAS reading on a level too small for the boxes (b does not divide N_l, or a subdomain's b + 2o + 1
// face columns would wrap onto themselves): the box clipped to the periodic level is the whole level, and
// its local solve the exact level solve with the gauge-fixed pseudo-inverse (as for the coarsest level).
bool ras_wraps(int N, int b, int o) { return N % b != 0 || b + 2 * o + 1 > N; }

// exact level solve of level l: L_l (from the stencils and the dense IB operator of its windows) + Z Z^T,
// inverted by the blocked Gauss-Jordan, minus Z Z^T.  Temporaries go to `tmp`, freed by the caller.
void ras_exact_setup(sib_ctx* c, int l, std::vector<void*>& tmp, int* ginfo, cudaStream_t s) {
    Level& lv = c->L[l];
    const int N = lv.N, n0 = N * N, n = 3 * n0;
    double* Bd = (double*)dalloc(c, sizeof(double) * 2 * (size_t)n0 * n0);
    double* Aug = (double*)dalloc(c, sizeof(double) * (size_t)n * 2 * n);
    void* work = dalloc(c, gauss_jordan_work_bytes(n));
    int* piv = (int*)dalloc(c, sizeof(int) * (size_t)n);
    tmp.insert(tmp.end(), {Bd, Aug, work, piv});
    CK(cudaMemsetAsync(Bd, 0, sizeof(double) * 2 * (size_t)n0 * n0, s));
    if (c->haveIB)
        KL(c, launch_window_dense((const double*)lv.win[0], lv.tiles, lv.hnTiles, N, lv.tx, lv.ty, lv.ntx, Bd, s));
    KL(c, launch_assemble_L0(N, c->rho, c->mu, c->dt, Bd, Aug, s));
    KL(c, launch_gauss_jordan(Aug, n, ginfo, piv, work, s));
    dfree(c, lv.rasPinv);
    lv.rasPinv = (double*)dalloc(c, sizeof(double) * (size_t)n * n);
    KL(c, launch_extract_pinv(Aug, piv, n, N, c->rho, lv.rasPinv, s));
    c->launches += 3;
}

// 16 x 16 boxes on level l: the full shared inverse by the blocked Gauss-Jordan, its tensor-core packs,
// and the Woodbury data of the level's nIB IB boxes (listed in lv.rasList)
void ras_huge_setup(sib_ctx* c, int l, int nIB, std::vector<void*>& tmp, int* ginfo, cudaStream_t s) {
    Level& lv = c->L[l];
    const int b = c->opts.box, o = c->opts.box_overlap;
    const int ne = ras_ne(b, o), n = ras_huge_n(b, o);
    double* Aug = (double*)dalloc(c, sizeof(double) * (size_t)n * 2 * n);
    void* work = dalloc(c, gauss_jordan_work_bytes(n));
    int* piv = (int*)dalloc(c, sizeof(int) * (size_t)n);
    tmp.insert(tmp.end(), {Aug, work, piv});
    const double h = lv.h, a0 = c->rho / c->dt + 4.0 * c->mu / (h * h), cc = c->mu / (h * h);
    KL(c, launch_ras_huge_assemble(lv.N, b, o, a0, cc, 1.0 / h, Aug, s));
    KL(c, launch_gauss_jordan(Aug, n, ginfo, piv, work, s));
    for (int p = 0; p < 2; ++p) dfree(c, lv.hugeInv[p]);
    lv.hugeInv[0] = dalloc(c, sizeof(double) * (size_t)ne * ne);
    lv.hugeInv[1] = dalloc(c, sizeof(float) * (size_t)ne * ne);
    KL(c, launch_ras_huge_extract(Aug, piv, b, o, (double*)lv.hugeInv[0], (float*)lv.hugeInv[1], s));
    const size_t gf = ras_tc_group_floats(b, o);
    const int groups = 3 * b * b / RAS_TC_GROUP;
    dfree(c, lv.rasTC);
    lv.rasTC = (float*)dalloc(c, sizeof(float) * gf * groups);
    lv.rasTCCap = gf * groups;
    for (int g = 0; g < groups; ++g) KL(c, launch_ras_tc_pack_rows(b, o, (const double*)lv.hugeInv[0], g, lv.rasTC + g * gf, s));
    c->launches += 3 + groups;
    lv.rasNIB = nIB;
    dfree(c, lv.wbOffT);
    dfree(c, lv.wbT);
    dfree(c, lv.wbOffW);
    dfree(c, lv.wbW);
    dfree(c, lv.wbScratch);
    lv.wbScratch = nullptr;
    lv.wbOffT = nullptr;
    lv.wbT = nullptr;
    lv.wbOffW = nullptr;
    lv.wbW = nullptr;
    lv.wbMmax = 0;
    if (nIB == 0) return;
    const RasIB ib{lv.slotOf, (const double*)lv.win[0], lv.tx, lv.ty, lv.ntx};
    int* dcnt = (int*)dalloc(c, sizeof(int) * (size_t)nIB);
    tmp.push_back(dcnt);
    KL(c, launch_ras_wb_count(lv.N, b, o, ib, lv.rasList, nIB, dcnt, s));
    std::vector<int> cnt(nIB), offT(nIB + 1, 0);
    std::vector<long long> offW(nIB, 0);
    CK(cudaMemcpyAsync(cnt.data(), dcnt, sizeof(int) * (size_t)nIB, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    long long wTot = 0;
    for (int k = 0; k < nIB; ++k) {
        offT[k + 1] = offT[k] + cnt[k];
        offW[k] = wTot;
        wTot += (long long)cnt[k] * cnt[k];
        lv.wbMmax = std::max(lv.wbMmax, cnt[k]);
    }
    lv.wbOffT = (int*)dalloc(c, sizeof(int) * (size_t)(nIB + 1));
    lv.wbOffW = (long long*)dalloc(c, sizeof(long long) * (size_t)nIB);
    lv.wbT = (int*)dalloc(c, sizeof(int) * (size_t)std::max(1, offT[nIB]));
    lv.wbW = (double*)dalloc(c, sizeof(double) * (size_t)std::max(1LL, wTot));
    lv.wbScratch = (double*)dalloc(c, sizeof(double) * (2 * (size_t)std::max(1, lv.wbMmax) + 3 * (size_t)b * b) * nIB);
    double* wwork = (double*)dalloc(c, sizeof(double) * (size_t)std::max(1LL, 2 * wTot));
    tmp.push_back(wwork);
    CK(cudaMemcpyAsync(lv.wbOffT, offT.data(), sizeof(int) * (size_t)(nIB + 1), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(lv.wbOffW, offW.data(), sizeof(long long) * (size_t)nIB, cudaMemcpyHostToDevice, s));
    KL(c, launch_ras_wb_fill(lv.N, b, o, ib, lv.rasList, nIB, lv.wbOffT, lv.wbT, s));
    KL(c, launch_ras_wb_setup(lv.N, b, o, ib, c->dt, lv.rasList, nIB, lv.wbOffT, lv.wbT, lv.wbOffW,
                              (const double*)lv.hugeInv[0], wwork, lv.wbW, c->rasInfo, lv.wbMmax, RAS_WB_ONE_MAX, s));
    // boxes with many IB-touched dofs: their [I + E Q | E] by the blocked Gauss-Jordan over the whole GPU,
    // one box after another (one block per box would leave each |T|^3 elimination to a single SM)
    int bigMax = 0;
    for (int k = 0; k < nIB; ++k)
        if (cnt[k] > RAS_WB_ONE_MAX) bigMax = std::max(bigMax, cnt[k]);
    if (bigMax > 0) {
        const int m16 = (bigMax + 15) / 16 * 16;
        double* augB = (double*)dalloc(c, sizeof(double) * (size_t)m16 * 2 * m16);
        int* pivB = (int*)dalloc(c, sizeof(int) * (size_t)m16);
        void* workB = dalloc(c, gauss_jordan_work_bytes(m16));
        tmp.insert(tmp.end(), {augB, pivB, workB});
        for (int k = 0; k < nIB; ++k)
            if (cnt[k] > RAS_WB_ONE_MAX) {
                launch_ras_wb_big(wwork + 2 * offW[k], cnt[k], augB, pivB, workB, c->rasInfo, lv.wbW + offW[k], s);
                c->launches += 2 + 3 * ((cnt[k] + 15) / 16);
            }
    }
    CK(cudaStreamSynchronize(s));   // the host vectors above are the copies' sources
    c->launches += 3;
}

void ras_setup_all(sib_ctx* c, cudaStream_t s) {
    const int b = c->opts.box, o = c->opts.box_overlap;
    const int ne = ras_ne(b, o), nown = 3 * b * b;
    const bool huge = ras_huge(b);
    const bool big = !huge && ras_big(b, o);
    const size_t matBytes = sizeof(double) * (size_t)ne * ne;
    std::vector<int> cnt(c->lmax + 1, 0);
    for (int l = 1; l <= c->lmax; ++l) {
        Level& lv = c->L[l];
        lv.rasExact = ras_wraps(lv.N, b, o);
        if (lv.rasExact) continue;
        if (c->haveIB && !lv.useWindow)
            throw SibError(SIB_ERR_UNIMPLEMENTED, "the box smoother needs the assembled IB windows on every level");
        const int nboxes = (lv.N / b) * (lv.N / b);
        if (nboxes > lv.rasBoxCap) {
            dfree(c, lv.rasList);
            dfree(c, lv.rasSlot);
            lv.rasList = (int*)dalloc(c, sizeof(int) * nboxes);
            lv.rasSlot = (int*)dalloc(c, sizeof(int) * nboxes);
            lv.rasBoxCap = nboxes;
        }
        if (!lv.rasCount) lv.rasCount = (int*)dalloc(c, sizeof(int));
        const RasIB ib{c->haveIB ? lv.slotOf : nullptr, (const double*)lv.win[0], lv.tx, lv.ty, lv.ntx};
        launch_ras_classify(lv.N, b, o, ib, lv.rasList, lv.rasCount, s);
        if (ib.slotOf) ++c->launches;
        CK(cudaMemcpyAsync(&cnt[l], lv.rasCount, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    CK(cudaMemsetAsync(c->rasInfo, 0, sizeof(int), s));
    std::vector<void*> tmp;   // set-up temporaries, freed at the end
    int* ginfo = (int*)dalloc(c, sizeof(int));
    tmp.push_back(ginfo);
    CK(cudaMemsetAsync(ginfo, 0, sizeof(int), s));
    int batch = 0;   // wide subdomains: matrices per set-up launch
    double* work = nullptr;
    if (big) {
        int most = 1;
        for (int l = 1; l <= c->lmax; ++l) most = std::max(most, 1 + cnt[l]);
        batch = (int)std::max<size_t>(1, std::min<size_t>((size_t)most, RAS_WORK_BYTES / matBytes));
        work = (double*)dalloc(c, matBytes * batch);
        tmp.push_back(work);
    }
    for (int l = 1; l <= c->lmax; ++l) {
        Level& lv = c->L[l];
        if (lv.rasExact) {
            ras_exact_setup(c, l, tmp, ginfo, s);
            continue;
        }
        const int nboxes = (lv.N / b) * (lv.N / b);
        launch_box_slots(nboxes, lv.rasList, lv.rasCount, lv.rasSlot, s);
        ++c->launches;
        if (huge) {
            ras_huge_setup(c, l, cnt[l], tmp, ginfo, s);
            continue;
        }
        const size_t ent = (size_t)(1 + cnt[l]) * ne * nown;
        if (ent > lv.rasInvCap) {
            dfree(c, lv.rasInv[0]);
            dfree(c, lv.rasInv[1]);
            lv.rasInv[0] = dalloc(c, sizeof(double) * ent);
            lv.rasInv[1] = dalloc(c, sizeof(float) * ent);
            lv.rasInvCap = ent;
        }
        const RasIB ib{c->haveIB ? lv.slotOf : nullptr, (const double*)lv.win[0], lv.tx, lv.ty, lv.ntx};
        lv.rasNIB = cnt[l];
        const double h = lv.h, a0 = c->rho / c->dt + 4.0 * c->mu / (h * h), cc = c->mu / (h * h);
        if (big) {
            for (int first = 0; first < 1 + cnt[l]; first += batch) {
                launch_ras_setup_big(lv.N, b, o, ib, a0, cc, 1.0 / h, c->dt, lv.rasList, first,
                                     std::min(batch, 1 + cnt[l] - first), work, (double*)lv.rasInv[0],
                                     (float*)lv.rasInv[1], c->rasInfo, s);
                ++c->launches;
            }
        } else {
            launch_ras_setup(lv.N, b, o, ib, a0, cc, 1.0 / h, c->dt, lv.rasList, cnt[l], (double*)lv.rasInv[0],
                             (float*)lv.rasInv[1], c->rasInfo, s);
            ++c->launches;
        }
        // the shared inverse (slot 0) packed for the tensor-core correction of FP32 levels
        const size_t pf = ras_tc_pack_floats(b, o);
        if (pf > lv.rasTCCap) {
            dfree(c, lv.rasTC);
            lv.rasTC = (float*)dalloc(c, sizeof(float) * pf);
            lv.rasTCCap = pf;
        }
        launch_ras_tc_pack(b, o, (const double*)lv.rasInv[0], lv.rasTC, s);
        ++c->launches;
    }
    int info = 0, gj = 0;
    CK(cudaMemcpyAsync(&info, c->rasInfo, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&gj, ginfo, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (void* p : tmp) dfree(c, p);
    kcheck(c);
    if (info != 0 || gj != 0) throw SibError(SIB_ERR_ARG, "a box subdomain operator is singular");
}

void setup(sib_ctx* c, cudaStream_t s) {
    CK(cudaEventRecord(c->ev0, s));
    invalidate_graphs(c);
    c->haveIB = c->M > 0 && c->E > 0;
    if (c->structDirty) {
        if (c->M > 0) {
            std::vector<int*> base(2 * (c->lmax + 1));
            std::vector<double*> w64(2 * (c->lmax + 1));
            std::vector<float*> w32(2 * (c->lmax + 1));
            for (int l = 0; l <= c->lmax; ++l)
                for (int q = 0; q < 2; ++q) {
                    base[2 * l + q] = c->L[l].base[q];
                    w64[2 * l + q] = (double*)c->L[l].p[0].w[q];
                    w32[2 * l + q] = (float*)c->L[l].p[1].w[q];
                }
            KL(c, launch_stencils(c->X, c->M, c->N, c->lmax, base.data(), w64.data(), w32.data(), s));
            KL(c, launch_deinterleave(c->X, c->M, c->Xc, s));
            int Mpad = 1;
            while (Mpad < c->M) Mpad <<= 1;
            c->Mpad = Mpad;
            for (int q = 0; q < 2; ++q) {
                KL(c, launch_sort_keys(c->L[c->lmax].base[q], c->M, Mpad, c->keys, s));
                launch_bitonic(c->keys, Mpad, s);
                KL(c, launch_unpack_sorted(c->keys, c->M, c->sorted[q], c->mkey[q], s));
                for (int l = 0; l <= c->lmax; ++l)
                    KL(c, launch_bins(c->mkey[q], c->M, c->L[l].N * c->L[l].N, 2 * (c->lmax - l),
                                      c->L[l].binStart[q], s));
            }
        }
        for (int l = 0; l <= c->lmax; ++l) {
            Level& lv = c->L[l];
            CK(cudaMemsetAsync(lv.tileFlag, 0, 2 * (size_t)lv.ntiles, s));
            if (c->M > 0)
                for (int q = 0; q < 2; ++q)
                    KL(c, launch_tile_flags(lv.base[q], c->M, lv.W, lv.N, lv.tx, lv.ty, lv.ntx, lv.tileFlag, s));
            KL(c, launch_tile_finish(lv.tileFlag, lv.ntx, lv.nty, lv.tiles, lv.nTiles, s));
            KL(c, launch_slot_map(lv.tiles, lv.nTiles, lv.ntiles, lv.slotOf, s));
            KL(c, launch_row_slots(lv.tileFlag, lv.tiles, lv.nTiles, lv.rowSlots, lv.nRowTiles, s));
        }
        launch_adjacency(c->edges, c->E, c->M, c->deg, c->adjStart, c->adjNbr, c->adjEid, s);
        std::vector<int> cnt(2 * (c->lmax + 1));
        for (int l = 0; l <= c->lmax; ++l) {
            CK(cudaMemcpyAsync(&cnt[2 * l], c->L[l].nTiles, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(&cnt[2 * l + 1], c->L[l].nRowTiles, sizeof(int), cudaMemcpyDeviceToHost, s));
        }
        CK(cudaStreamSynchronize(s));
        for (int l = 0; l <= c->lmax; ++l) {
            Level& lv = c->L[l];
            lv.hnTiles = cnt[2 * l];
            lv.hnRowTiles = cnt[2 * l + 1];
            if (lv.hnTiles > lv.winSlots || !lv.win[0]) {
                dfree(c, lv.win[0]);
                dfree(c, lv.win[1]);
                const size_t ent = (size_t)(lv.hnTiles > 0 ? lv.hnTiles : 1) * 2 * WIN_SIZE * lv.tx * lv.ty;
                lv.win[0] = dalloc(c, sizeof(double) * ent);
                lv.win[1] = dalloc(c, sizeof(float) * ent);
                lv.winSlots = lv.hnTiles > 0 ? lv.hnTiles : 1;
            }
            if (!lv.winOverflow) lv.winOverflow = (int*)dalloc(c, sizeof(int));
            // warp per face when a face gathers from many markers on average
            const double faces = (double)lv.hnTiles * lv.tx * lv.ty;
            lv.spreadWarp = faces > 0 && (double)c->M * lv.W * lv.W > 16.0 * faces ? 1 : 0;
        }
        kcheck(c);
        c->structDirty = false;
        c->kappaDirty = true;
    }
    if (c->kappaDirty) {
        KL(c, launch_adj_kappa<double>(c->adjEid, c->kappa, 2 * c->E, c->kap64, s));
        KL(c, launch_adj_kappa<float>(c->adjEid, c->kappa, 2 * c->E, c->kap32, s));
        // assembled windows of [S K J]^l: finest level from the markers, coarser levels by the
        // Galerkin product R_u B P_u of the next finer window; one overflow flag read back
        if (c->haveIB) {
            Level& lf = c->L[c->lmax];
            CK(cudaMemsetAsync(lf.winOverflow, 0, sizeof(int), s));
            KL(c, launch_kj_patch(ibk<double>(c, c->lmax), c->adjStart, c->adjNbr, c->kap64, c->KJ, lf.winOverflow, s));
            KL(c, launch_window_fine(ibk<double>(c, c->lmax), c->KJ, lf.tiles, lf.hnTiles, lf.tx, lf.ty, lf.ntx,
                                     (double*)lf.win[0], s));
            // the cavity's Galerkin product uses P_u restricted to the unknowns: every level's windows
            // lose their wall couplings before the next coarser product
            if (cavity(c))
                KL(c, launch_cavity_mask_windows((double*)lf.win[0], lf.tiles, lf.hnTiles, lf.N, lf.tx, lf.ty, lf.ntx, s));
            for (int l = c->lmax - 1; l >= 0; --l) {
                Level& F = c->L[l + 1];
                Level& C = c->L[l];
                KL(c, launch_window_rap((const double*)F.win[0], F.slotOf, F.N, F.tx, F.ty, F.ntx, C.tiles, C.hnTiles, C.N,
                                        C.tx, C.ty, C.ntx, (double*)C.win[0], s));
                if (cavity(c))
                    KL(c, launch_cavity_mask_windows((double*)C.win[0], C.tiles, C.hnTiles, C.N, C.tx, C.ty, C.ntx, s));
            }
            int ovf = 0;
            CK(cudaMemcpyAsync(&ovf, lf.winOverflow, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int l = 0; l <= c->lmax; ++l) c->L[l].useWindow = ovf == 0;
        } else {
            for (int l = 0; l <= c->lmax; ++l) c->L[l].useWindow = 0;
        }
        for (int l = 0; l <= c->lmax; ++l) {
            Level& lv = c->L[l];
            const size_t n = (size_t)lv.N * lv.N;
            for (int pi = 0; pi < 2; ++pi) {
                const size_t e = pi == 0 ? 8 : 4;
                CK(cudaMemsetAsync(lv.p[pi].fib, 0, e * 2 * n, s));
            }
            CK(cudaMemsetAsync(lv.p[0].ibd, 0, 8 * 4 * n, s));
            if (c->haveIB && l > 0) {
                if (lv.useWindow)
                    KL(c, launch_window_patch((const double*)lv.win[0], lv.tiles, lv.hnTiles, lv.N, lv.tx, lv.ty, lv.ntx,
                                              (double*)lv.p[0].ibd, s));
                else
                    KL(c, launch_patch_entries(ibk<double>(c, l), c->adjStart, c->adjNbr, c->kap64, lv.tiles,
                                               lv.rowSlots, lv.nRowTiles, lv.hnRowTiles, lv.tx, lv.ty, lv.ntx,
                                               (double*)lv.p[0].ibd, s));
            }
            KL(c, (launch_convert<double, float>((const double*)lv.p[0].ibd, (float*)lv.p[1].ibd, 4 * (int64_t)n,
                                                 s)));
            if (lv.useWindow) {
                const int64_t ent = (int64_t)lv.hnTiles * 2 * WIN_SIZE * lv.tx * lv.ty;
                KL(c, (launch_convert<double, float>((const double*)lv.win[0], (float*)lv.win[1], ent, s)));
            }
            // the solve applies the windows on coarse levels, and on the finest level when the
            // windows hold fewer than 8 coefficients per marker-face pair of the marker path
            const double winEnt = (double)lv.hnTiles * lv.tx * lv.ty * 2.0 * WIN_SIZE;
            const double pairs = (double)c->M * 2.0 * lv.W * lv.W;
            lv.applyWindow = c->haveIB && lv.useWindow && (l < c->lmax || winEnt <= 8.0 * pairs);
            lv.spReady = false;
            if (c->haveIB && !lv.applyWindow && lv.hnRowTiles > 0) {   // the marker path's stored spreading
                const size_t rows = 2 * (size_t)lv.hnRowTiles * lv.tx * lv.ty;
                const size_t ent = 2 * (size_t)c->M * lv.W * lv.W;
                if (rows > lv.spRowsCap) {
                    for (void* p : {(void*)lv.spLoc, (void*)lv.spOff, (void*)lv.spTileCnt, (void*)lv.spTileOff})
                        dfree(c, p);
                    lv.spLoc = (int*)dalloc(c, sizeof(int) * rows);
                    lv.spOff = (int*)dalloc(c, sizeof(int) * (rows + 1));
                    lv.spTileCnt = (int*)dalloc(c, sizeof(int) * 2 * (size_t)lv.hnRowTiles);
                    lv.spTileOff = (int*)dalloc(c, sizeof(int) * (2 * (size_t)lv.hnRowTiles + 1));
                    lv.spRowsCap = rows;
                }
                if (ent > lv.spEntCap) {
                    for (void* p : {(void*)lv.spCol, (void*)lv.spV64, (void*)lv.spV32}) dfree(c, p);
                    lv.spCol = (int*)dalloc(c, sizeof(int) * ent);
                    lv.spV64 = (double*)dalloc(c, sizeof(double) * ent);
                    lv.spV32 = (float*)dalloc(c, sizeof(float) * ent);
                    lv.spEntCap = ent;
                }
                c->launches += 3;
                launch_spread_store(ibk<double>(c, l), (const float*)lv.p[1].w[0], (const float*)lv.p[1].w[1], lv.tiles,
                                    lv.rowSlots, lv.nRowTiles, lv.hnRowTiles, lv.tx, lv.ty, lv.ntx, lv.spLoc,
                                    lv.spTileCnt, lv.spTileOff, (int64_t)ent, lv.spOff, lv.spCol, lv.spV64, lv.spV32,
                                    s);
                lv.spReady = true;
            }
        }
        Level& l0 = c->L[0];
        CK(cudaMemsetAsync(c->B0, 0, sizeof(double) * 2 * (size_t)c->n0 / 3 * c->n0 / 3, s));
        if (c->haveIB) {
            if (l0.useWindow)
                KL(c, launch_window_dense((const double*)l0.win[0], l0.tiles, l0.hnTiles, l0.N, l0.tx, l0.ty, l0.ntx,
                                          c->B0, s));
            else
                KL(c, launch_dense_ib(ibk<double>(c, 0), c->adjStart, c->adjNbr, c->kap64, c->B0, s));
        }
        c->kappaDirty = false;
        c->fluidDirty = true;
    }
    // coarsest pseudo-inverse (depends on rho, mu, dt and kappa).  The Gauss-Jordan inversion holds
    // one 16-block cluster for about a millisecond; it runs on the auxiliary stream, beside the SC
    // eigenvalue estimates below (which do not use it), and the main stream joins it at the end.
    {
        const int n = c->n0;
        if (cavity(c))
            KL(c, launch_cavity_assemble_L0(c->L[0].N, c->rho, c->mu, c->dt, c->B0, c->Aug, s));
        else
            KL(c, launch_assemble_L0(c->L[0].N, c->rho, c->mu, c->dt, c->B0, c->Aug, s));
        CK(cudaEventRecord(c->evFork, s));
        CK(cudaStreamWaitEvent(c->aux, c->evFork, 0));
        KL(c, launch_gauss_jordan(c->Aug, n, c->info, c->piv, c->gjWork, c->aux));
        // the gauge's Z Z^T comes off the pressure block alone in the cavity (passed as rho != 0)
        KL(c, launch_extract_pinv(c->Aug, c->piv, n, c->L[0].N, cavity(c) ? 1.0 : c->rho, c->Pinv, c->aux));
        CK(cudaEventRecord(c->evJoin, c->aux));
    }
    // Vanka patch factors (they depend on the fluid parameters and the patch entries)
    for (int l = 1; l <= c->lmax; ++l) {
        Level& lv = c->L[l];
        const int64_t n7 = 7LL * lv.N * lv.N;
        KL(c, launch_patch_factors(gridk<double>(c, l), (double*)lv.p[0].pf, s));
        KL(c, (launch_convert<double, float>((const double*)lv.p[0].pf, (float*)lv.p[1].pf, n7, s)));
    }
    if (c->opts.smoother == SIB_SMOOTHER_RAS && c->lmax > 0) ras_setup_all(c, s);
    if (cavity(c))   // the cavity sweep's patch corrections, allocated outside any graph capture
        for (int l = 1; l <= c->lmax; ++l)
            for (int pi = 0; pi < 2; ++pi)
                if (!c->L[l].p[pi].cav)
                    c->L[l].p[pi].cav = dalloc(c, (pi == 0 ? 8 : 4) * 5 * (size_t)c->L[l].N * c->L[l].N);
    if (c->opts.smoother == SIB_SMOOTHER_SC) {
        alloc_sc_bufs(c);
        for (int l = 1; l <= c->lmax; ++l) {
            Level& lv = c->L[l];
            if (c->lamOverride) {
                lv.lamA = c->lamA_ov[l];
                lv.lamM = c->lamM_ov[l];
            }
        }
        for (int l = 1; l <= c->lmax; ++l) {
            Level& lv = c->L[l];
            const int64_t n3 = 3LL * lv.N * lv.N;
            KL(c, launch_sc_diag(gridk<double>(c, l), (double*)lv.p[0].dinv, s));
            KL(c, (launch_convert<double, float>((const double*)lv.p[0].dinv, (float*)lv.p[1].dinv, n3, s)));
        }
        if (!c->lamOverride && c->lmax > 0) {
            const int L = c->lmax;
            // the levels' chains side by side: a level on its own stream, except where the IB force
            // goes through the markers (the marker buffers are shared), which stays on s in order
            auto levels = [&](auto enqueue) {
                CK(cudaEventRecord(c->evFork, s));
                for (int l = 1; l <= L; ++l) {
                    const bool own = (!c->haveIB || c->L[l].applyWindow) && l < sib_ctx::LVS && c->lvStream[l];
                    cudaStream_t ls = own ? c->lvStream[l] : s;
                    if (own) CK(cudaStreamWaitEvent(ls, c->evFork, 0));
                    enqueue(l, c->part + (size_t)l * NBLK, ls);
                    if (own) CK(cudaEventRecord(c->lvDone[l], ls));
                }
                for (int l = 1; l <= L; ++l)
                    if ((!c->haveIB || c->L[l].applyWindow) && l < sib_ctx::LVS && c->lvStream[l])
                        CK(cudaStreamWaitEvent(s, c->lvDone[l], 0));
            };
            levels([&](int l, double* part, cudaStream_t ls) { power_A_enqueue(c, l, 300 + l, part, ls); });
            CK(cudaMemcpyAsync(c->hbuf + 300, c->scal + 300, sizeof(double) * 60, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int l = 1; l <= L; ++l) c->L[l].lamA = std::sqrt(c->hbuf[300 + l] / c->hbuf[340 + l]);
            levels([&](int l, double* part, cudaStream_t ls) { power_M_enqueue(c, l, 320 + l, part, ls); });
            CK(cudaMemcpyAsync(c->hbuf + 320, c->scal + 320, sizeof(double) * 60, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int l = 1; l <= L; ++l) c->L[l].lamM = std::sqrt(c->hbuf[320 + l] / c->hbuf[360 + l]);
        }
    }
    CK(cudaStreamWaitEvent(s, c->evJoin, 0));
    {
        int info = 0;
        CK(cudaMemcpyAsync(&info, c->info, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (info != 0) throw SibError(SIB_ERR_ARG, "coarsest operator is singular beyond its gauge kernel");
        c->fluidDirty = false;
    }
    alloc_krylov(c);
    CK(cudaEventRecord(c->ev1, s));
    CK(cudaStreamSynchronize(s));
    kcheck(c);
    float ms = 0;
    cudaEventElapsedTime(&ms, c->ev0, c->ev1);
    c->setup_ms = ms;
    c->setupDone = true;
}

void require_setup(sib_ctx* c) {
    if (!c->setupDone || c->structDirty || c->kappaDirty || c->fluidDirty)
        throw SibError(SIB_ERR_STATE, "sib_setup must be called after the last change of fluid, structure or kappa");
}

// ---- flexible GMRES (right-preconditioned, CGS2, Givens) ---------------------------------------
void dot(sib_ctx* c, const double* x, const double* y, int64_t n, double* dst, cudaStream_t s) { dot_into(c, x, y, n, dst, s); }

void project(sib_ctx* c, double* x, cudaStream_t s) {
    // kernel of the operator: the constant pressure, and for rho = 0 on the periodic grid the
    // constant velocities too (the cavity's walls fix the velocity)
    const int mask = c->rho == 0.0 && !cavity(c) ? 7 : 4;
    KL(c, launch_block_means(x, c->N, 3, c->part, NBLK, s));
    KL(c, launch_subtract_means(x, c->N, c->part, NBLK, mask, s));
}

// z = M^{-1} v (V-cycle in the configured precision, casts fused into the copies)
void precondition(sib_ctx* c, const double* v, double* z, cudaStream_t s) {
    const int64_t n = n3f(c);
    Level& lv = c->L[c->lmax];
    if (c->opts.vcycle_fp32) {
        KL(c, (launch_convert<double, float>(v, (float*)lv.p[1].b, n, s)));
        float* out = vcycle<float>(c, s);
        KL(c, (launch_convert<float, double>(out, z, n, s)));
    } else {
        KL(c, (launch_convert<double, double>(v, (double*)lv.p[0].b, n, s)));
        double* out = vcycle<double>(c, s);
        KL(c, (launch_convert<double, double>(out, z, n, s)));
    }
}

void matvec(sib_ctx* c, const double* x, double* y, cudaStream_t s) { apply_operator<double>(c, c->lmax, x, nullptr, y, s); }

int fgmres(sib_ctx* c, const double* b, double* x, sib_stats* st, cudaStream_t s) {
    const int64_t n = n3f(c);
    const int max_it = c->opts.max_it;
    const int mres = c->mcap;
    double* hb = c->hbuf;
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    dot(c, b, b, n, c->scal + 256, s);
    CK(cudaMemcpyAsync(hb, c->scal + 256, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double bnorm = std::sqrt(hb[0]);
    if (!std::isfinite(bnorm)) throw SibError(SIB_ERR_NONFINITE, "right-hand side is not finite");
    std::vector<double> hist;
    hist.push_back(bnorm);
    int its = 0;
    bool converged = bnorm == 0.0;
    double est = bnorm;
    std::vector<double> H((size_t)(mres + 1) * mres), cs(mres), sn(mres), g(mres + 1), y(mres);
    while (!converged && its < max_it) {
        double* r = c->V;   // V_0
        double beta;
        if (its == 0) {
            KL(c, (launch_convert<double, double>(b, r, n, s)));
            beta = bnorm;
        } else {
            matvec(c, x, c->res, s);
            KL(c, launch_axpby<double>(1.0, b, -1.0, c->res, r, n, s));
            dot(c, r, r, n, c->scal + 256, s);
            CK(cudaMemcpyAsync(hb, c->scal + 256, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            beta = std::sqrt(hb[0]);
        }
        if (beta == 0.0) {
            converged = true;
            break;
        }
        // scale V0 by 1/beta (scal[258] = beta^2, staged through pinned memory)
        hb[450] = beta * beta;
        CK(cudaMemcpyAsync(c->scal + 258, hb + 450, sizeof(double), cudaMemcpyHostToDevice, s));
        KL(c, launch_scale(r, c->scal, 258, n, s));
        const int m = std::min(mres, max_it - its);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double* vj = c->V + (int64_t)j * n;
            double* zj = c->Z + (int64_t)j * n;
            double* w = c->V + (int64_t)(j + 1) * n;
            precondition(c, vj, zj, s);
            matvec(c, zj, w, s);
            KL(c, launch_multidot(c->V, n, j + 1, w, n, c->part, NBLK, s));
            KL(c, launch_reduce_partials(c->part, j + 1, NBLK, c->scal, s));
            KL(c, launch_multi_axpy(c->V, n, j + 1, c->scal, -1.0, w, n, s));
            KL(c, launch_multidot(c->V, n, j + 1, w, n, c->part, NBLK, s));
            KL(c, launch_reduce_partials(c->part, j + 1, NBLK, c->scal + 128, s));
            KL(c, launch_multi_axpy(c->V, n, j + 1, c->scal + 128, -1.0, w, n, s));
            dot(c, w, w, n, c->scal + 256, s);
            KL(c, launch_scale(w, c->scal, 256, n, s));
            CK(cudaMemcpyAsync(hb, c->scal, sizeof(double) * 257, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            double* Hj = &H[(size_t)j * (mres + 1)];   // column j
            for (int i = 0; i <= j; ++i) Hj[i] = hb[i] + hb[128 + i];
            const double hn = std::sqrt(hb[256]);
            Hj[j + 1] = hn;
            for (int i = 0; i < j; ++i) {
                const double a = Hj[i], bq = Hj[i + 1];
                Hj[i] = cs[i] * a + sn[i] * bq;
                Hj[i + 1] = -sn[i] * a + cs[i] * bq;
            }
            const double d = std::hypot(Hj[j], Hj[j + 1]);
            cs[j] = Hj[j] / d;
            sn[j] = Hj[j + 1] / d;
            Hj[j] = d;
            Hj[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++its;
            k = j + 1;
            est = std::fabs(g[j + 1]);
            hist.push_back(est);
            if (!std::isfinite(est) || !std::isfinite(d)) throw SibError(SIB_ERR_NONFINITE, "non-finite value in FGMRES");
            if (est <= c->opts.rtol * bnorm || hn == 0.0) {
                converged = true;
                break;
            }
            if (its >= max_it) break;
        }
        for (int i = k - 1; i >= 0; --i) {
            double acc = g[i];
            for (int q = i + 1; q < k; ++q) acc -= H[(size_t)q * (mres + 1) + i] * y[q];
            y[i] = acc / H[(size_t)i * (mres + 1) + i];
        }
        for (int i = 0; i < k; ++i) hb[300 + i] = y[i];
        CK(cudaMemcpyAsync(c->scal + 384, hb + 300, sizeof(double) * k, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));   // hb is reused by the next cycle's reads
        KL(c, launch_multi_axpy(c->Z, n, k, c->scal + 384, 1.0, x, n, s));
    }
    project(c, x, s);
    // true residual of the gauge-fixed solution
    matvec(c, x, c->res, s);
    KL(c, launch_axpby<double>(1.0, b, -1.0, c->res, c->res, n, s));
    dot(c, c->res, c->res, n, c->scal + 256, s);
    CK(cudaMemcpyAsync(hb, c->scal + 256, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double rt = std::sqrt(hb[0]);
    if (st) {
        st->iterations = its;
        st->converged = converged ? 1 : 0;
        st->bnorm = bnorm;
        st->rel_residual = bnorm > 0 ? rt / bnorm : 0.0;
        st->rel_residual_est = bnorm > 0 ? est / bnorm : 0.0;
        const size_t nh = std::min<size_t>(hist.size(), 101);
        for (size_t i = 0; i < nh; ++i) st->history[i] = hist[i];
    }
    return converged ? SIB_OK : SIB_ERR_NOT_CONVERGED;
}

// ---- device-side FGMRES cycle: a conditional WHILE graph node runs the iterations -------------
template <typename T>
void build_fg_graph(sib_ctx* c) {
    const int pi = Prec<T>::id;
    const int64_t n = n3f(c);
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    const int64_t before = c->launches;
    try {
        cudaGraphConditionalHandle h;
        CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t wnode;
        CK(cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &p));
        cudaGraph_t body = p.conditional.phGraph_out[0];
        cudaStream_t s = c->cap;
        apply_l2_policy(c);
        CK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        try {
            Level& lv = c->L[c->lmax];
            // V_j (stored from the previous step's w), the V-cycle, z_j, w = L z_j, two classical
            // Gram-Schmidt passes (the second also gives ||w||^2), the Hessenberg column and the
            // loop decision
            KL(c, launch_fg_prep<T>(c->V, c->res, n, c->fg, (T*)lv.p[pi].b, s));
            T* out = vcycle_level<T>(c, c->lmax, s);
            KL(c, launch_fg_zstore<T>(out, c->Z, n, c->fg, c->zcur, s));
            matvec(c, c->zcur, c->res, s);
            KL(c, launch_multidot_dev(c->V, n, c->res, n, c->part, c->fg, s));
            KL(c, launch_reduce_partials_dev(c->part, 0, c->scal, c->fg, 0, s));
            KL(c, launch_multi_axpy_dev(c->V, n, c->scal, -1.0, c->res, n, c->fg, 0, s));
            KL(c, launch_multidot_dev(c->V, n, c->res, n, c->part, c->fg, s));
            KL(c, launch_reduce_partials_dev(c->part, 0, c->scal + 128, c->fg, 0, s));
            int nb = 0;
            KL(c, nb = launch_multi_axpy_norm_dev(c->V, n, c->scal + 128, -1.0, c->res, n, c->fg, c->part, s));
            KL(c, launch_reduce_partials_dev(c->part, nb, c->scal + 256, c->fg, 1, s));
            KL(c, launch_fg_arnoldi(c->fg, c->scal, c->scal + 128, c->scal + 256, h, s));
        } catch (...) {
            cudaGraph_t tmp;
            cudaStreamEndCapture(s, &tmp);
            throw;
        }
        cudaGraph_t tmp;
        CK(cudaStreamEndCapture(s, &tmp));
        const int64_t mid = c->launches;
        CK(cudaStreamBeginCaptureToGraph(s, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
        const double* y = reinterpret_cast<const double*>(reinterpret_cast<const char*>(c->fg) + offsetof(FgDev, y));
        KL(c, launch_fg_backsolve(c->fg, s));
        KL(c, launch_multi_axpy_dev(c->Z, n, y, 1.0, c->sol, n, c->fg, 1, s));
        CK(cudaStreamEndCapture(s, &tmp));
        CK(cudaGraphInstantiate(&c->fgExec[pi], g, 0));
        c->fgBody[pi] = mid - before;
        c->fgTail[pi] = c->launches - mid;
    } catch (...) {
        c->launches = before;
        cudaGraphDestroy(g);
        cudaGetLastError();
        throw;
    }
    c->launches = before;
    cudaGraphDestroy(g);
}

// FGMRES with the cycles on the device; x is accumulated in c->sol.  Synchronises once per cycle.
int fgmres_device(sib_ctx* c, const double* b, double* w, sib_stats* st, cudaStream_t s) {
    const int64_t n = n3f(c);
    const int max_it = c->opts.max_it;
    const int pi = c->opts.vcycle_fp32 ? 1 : 0;
    double* hb = c->hbuf;
    double* x = c->sol;
    if (!c->fgExec[pi]) {
        if (pi == 1)
            build_fg_graph<float>(c);
        else
            build_fg_graph<double>(c);
    }
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    dot(c, b, b, n, c->scal + 256, s);
    CK(cudaMemcpyAsync(hb, c->scal + 256, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double bnorm = std::sqrt(hb[0]);
    if (!std::isfinite(bnorm)) throw SibError(SIB_ERR_NONFINITE, "right-hand side is not finite");
    std::vector<double> hist{bnorm};
    int its = 0;
    bool converged = bnorm == 0.0;
    double est = bnorm;
    while (!converged && its < max_it) {
        double* r = c->V;
        double beta;
        if (its == 0) {
            KL(c, (launch_convert<double, double>(b, r, n, s)));
            beta = bnorm;
        } else {
            matvec(c, x, c->res, s);
            KL(c, launch_axpby<double>(1.0, b, -1.0, c->res, r, n, s));
            dot(c, r, r, n, c->scal + 256, s);
            CK(cudaMemcpyAsync(hb, c->scal + 256, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            beta = std::sqrt(hb[0]);
        }
        if (beta == 0.0) {
            converged = true;
            break;
        }
        hb[450] = beta * beta;
        CK(cudaMemcpyAsync(c->scal + 258, hb + 450, sizeof(double), cudaMemcpyHostToDevice, s));
        KL(c, launch_scale(r, c->scal, 258, n, s));
        const int m = std::min(c->mcap, max_it - its);
        KL(c, launch_fg_init(c->fg, beta, m, m, c->opts.rtol * bnorm, s));
        CK(cudaGraphLaunch(c->fgExec[pi], s));
        // cycle results: the int header (j, jn, its, k, converged, ...) and (tol, est, ...)
        int hdr[8];
        double dv[4];
        CK(cudaMemcpyAsync(hdr, c->fg, sizeof(hdr), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(dv, reinterpret_cast<const char*>(c->fg) + offsetof(FgDev, tol), sizeof(dv),
                           cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hb + 300, reinterpret_cast<const char*>(c->fg) + offsetof(FgDev, hist),
                           sizeof(double) * (FG_MAXM + 1), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const int cyc = hdr[2];
        c->launches += (int64_t)cyc * c->fgBody[pi] + c->fgTail[pi];
        for (int i = 1; i <= cyc; ++i) hist.push_back(hb[300 + i]);
        its += cyc;
        est = dv[1];
        converged = hdr[4] != 0;
        if (!std::isfinite(est)) throw SibError(SIB_ERR_NONFINITE, "non-finite value in FGMRES");
        if (cyc == 0) break;
    }
    project(c, x, s);
    matvec(c, x, c->res, s);
    KL(c, launch_axpby<double>(1.0, b, -1.0, c->res, c->res, n, s));
    dot(c, c->res, c->res, n, c->scal + 256, s);
    CK(cudaMemcpyAsync(hb, c->scal + 256, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (w != x) CK(cudaMemcpyAsync(w, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    const double rt = std::sqrt(hb[0]);
    if (st) {
        st->iterations = its;
        st->converged = converged ? 1 : 0;
        st->bnorm = bnorm;
        st->rel_residual = bnorm > 0 ? rt / bnorm : 0.0;
        st->rel_residual_est = bnorm > 0 ? est / bnorm : 0.0;
        const size_t nh = std::min<size_t>(hist.size(), 101);
        for (size_t i = 0; i < nh; ++i) st->history[i] = hist[i];
    }
    return converged ? SIB_OK : SIB_ERR_NOT_CONVERGED;
}

// b = g (+ S K X^n), projected
void build_rhs(sib_ctx* c, const double* g, bool addSKX, cudaStream_t s) {
    const int64_t n = n3f(c);
    const int64_t nv = 2LL * c->N * c->N;
    KL(c, (launch_convert<double, double>(g, c->rhs, n, s)));
    if (addSKX && c->haveIB) {
        Level& lv = c->L[c->lmax];
        IBK<double> k = ibk<double>(c, c->lmax);
        double* F = (double*)c->F[0];
        KL(c, launch_spring<double>(c->adjStart, c->adjNbr, c->kap64, c->M, c->Xc, F, s));
        KL(c, launch_spread<double>(k, F, (double*)lv.p[0].fib, lv.tiles, lv.nTiles, lv.hnTiles, lv.tx, lv.ty, lv.ntx,
                                    lv.spreadWarp, s));
        KL(c, launch_axpby<double>(1.0, c->rhs, 1.0, (const double*)lv.p[0].fib, c->rhs, nv, s));
    }
    if (cavity(c)) {   // the walls are not unknowns; the moving lid enters through the ghost values
        KL(c, launch_cavity_zero_walls<double>(c->rhs, c->N, s));
        KL(c, launch_cavity_add_lid(c->rhs, c->N, c->mu, s));
    }
    project(c, c->rhs, s);
}

int solve_impl(sib_ctx* c, const double* g, double* w, sib_stats* st, cudaStream_t s, bool addSKX) {
    require_setup(c);
    CK(cudaMemsetAsync(c->flag, 0, sizeof(int), s));
    KL(c, launch_check_finite(g, n3f(c), c->flag, s));
    int fl = 0;
    CK(cudaMemcpyAsync(&fl, c->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (fl) throw SibError(SIB_ERR_NONFINITE, "right-hand side contains a non-finite value");
    CK(cudaEventRecord(c->ev0, s));
    build_rhs(c, g, addSKX, s);
    int rc;
    if (c->opts.use_graphs && !c->fgUnavailable && c->mcap <= FG_MAXM) {
        try {
            rc = fgmres_device(c, c->rhs, w, st, s);
        } catch (const SibError& e) {
            if (c->fgExec[0] || c->fgExec[1] || e.code != SIB_ERR_CUDA) throw;
            c->fgUnavailable = true;   // conditional graphs not supported here: host loop
            rc = fgmres(c, c->rhs, w, st, s);
        }
    } else {
        rc = fgmres(c, c->rhs, w, st, s);
    }
    CK(cudaEventRecord(c->ev1, s));
    CK(cudaEventSynchronize(c->ev1));
    kcheck(c);
    if (st) {
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        st->solve_ms = ms;
        st->setup_ms = c->setup_ms;
    }
    return rc;
}

bool valid_prec(int p) { return p == SIB_PREC_FP64 || p == SIB_PREC_FP32; }
void check_level(sib_ctx* c, int l, int lo) {
    if (l < lo || l > c->lmax) throw SibError(SIB_ERR_ARG, "level out of range");
}

template <typename T>
void smooth_impl(sib_ctx* c, int l, T* x, const T* b, int sweeps, cudaStream_t s) {
    Level& lv = c->L[l];
    const int pi = Prec<T>::id;
    const int64_t n3 = 3LL * lv.N * lv.N;
    T* xa = (T*)lv.p[pi].x;
    T* xb = (T*)lv.p[pi].xt;
    CK(cudaMemcpyAsync(xa, x, sizeof(T) * n3, cudaMemcpyDeviceToDevice, s));
    if (c->opts.smooth_krylov) {
        if (sweeps > 0) {
            wrapped_smooth<T>(c, l, (const T*)xa, b, xb, sweeps, s);
            std::swap(xa, xb);
        }
    } else {
        for (int k = 0; k < sweeps; ++k) {
            sweep<T>(c, l, xa, b, xb, s);
            std::swap(xa, xb);
        }
    }
    CK(cudaMemcpyAsync(x, xa, sizeof(T) * n3, cudaMemcpyDeviceToDevice, s));
}

template <typename T>
void time_kernel(sib_ctx* c, int kernel, int l, int reps, bool cold, cudaStream_t s, double* ms, double* bytes) {
    Level& lv = c->L[l];
    const int pi = Prec<T>::id;
    LevelBuf& b = lv.p[pi];
    const double n = (double)lv.N * lv.N;
    const double w = sizeof(T);
    const double active = c->haveIB ? (double)lv.hnTiles * lv.tx * lv.ty : 0.0;   // cells in IB-active tiles
    const int64_t n3 = 3LL * lv.N * lv.N;
    CK(cudaMemsetAsync(b.x, 0, sizeof(T) * n3, s));
    CK(cudaMemsetAsync(b.b, 0, sizeof(T) * n3, s));
    CK(cudaMemsetAsync(b.r, 0, sizeof(T) * n3, s));
    GridK<T> g = gridk<T>(c, l);
    IBK<T> k = ibk<T>(c, l);
    T* U = (T*)c->U[pi];
    T* F = (T*)c->F[pi];
    double by = 0;
    auto launch = [&]() {
        switch (kernel) {
            case SIB_KERNEL_VANKA:
                launch_vanka<T>(g, (const T*)b.x, (const T*)b.b, (T*)b.xt, s);
                break;
            case SIB_KERNEL_RESIDUAL:
                launch_residual<T>(g, (const T*)b.x, (const T*)b.b, (T*)b.r, s);
                break;
            case SIB_KERNEL_SPREAD:
                spread_apply<T>(c, lv, k, F, (T*)b.fib, s);
                break;
            case SIB_KERNEL_INTERP:
                launch_interp<T>(k, (const T*)b.x, U, s);
                break;
            case SIB_KERNEL_RESTRICT:
                launch_restrict<T>(c->L[l - 1].N, (const T*)b.r, (T*)c->L[l - 1].p[pi].b, s);
                break;
            case SIB_KERNEL_RESIDUAL_RESTRICT:
                launch_residual_restrict<T>(g, (const T*)b.x, (const T*)b.b, (T*)c->L[l - 1].p[pi].b, s);
                break;
            case SIB_KERNEL_PROLONG:
                launch_prolong_add<T>(c->L[l - 1].N, (const T*)c->L[l - 1].p[pi].x, (T*)b.x, s);
                break;
            case SIB_KERNEL_RAS:
                ras_apply<T>(c, l, (const T*)b.r, (const T*)b.x, (T*)b.xt, 1.0, s);
                break;
            case SIB_KERNEL_IB_WINDOW:
                launch_ib_window<T>((const T*)lv.win[pi], lv.tiles, lv.rowSlots, lv.nRowTiles, lv.hnRowTiles, lv.N,
                                    lv.tx, lv.ty, lv.ntx, (const T*)b.x, (T*)b.fib, s);
                break;
            default:
                throw SibError(SIB_ERR_ARG, "unknown kernel id");
        }
    };
    switch (kernel) {
        case SIB_KERNEL_VANKA:   // x, b read; xo written; fib (2) + patch factors (7) words in active tiles
            by = 9.0 * n * w + 9.0 * active * w;
            break;
        case SIB_KERNEL_RESIDUAL:
            by = 9.0 * n * w + 2.0 * active * w;
            break;
        case SIB_KERNEL_SPREAD: {   // every face of a stencil-touched tile written and its bin offset read, every
                                    // marker's weights, sorted id and force read once
            const double rows = c->haveIB ? (double)lv.hnRowTiles * lv.tx * lv.ty : 0.0;
            by = 2.0 * rows * w + (double)c->M * 2.0 * (8.0 * w + 4.0 + w) + 2.0 * rows * 4.0;
            break;
        }
        case SIB_KERNEL_INTERP:   // stencil origin, weights, W^2 velocities (distinct faces at most), U
            by = (double)c->M * 2.0 * (4.0 + 8.0 * w + w) + std::min(2.0 * active, (double)c->M * 2.0 * lv.W * lv.W) * w;
            break;
        case SIB_KERNEL_RESTRICT:
            by = 3.0 * n * w + 0.75 * n * w;
            break;
        case SIB_KERNEL_RESIDUAL_RESTRICT:   // x, b read; the coarse residual written; f_IB in active tiles
            by = 6.0 * n * w + 0.75 * n * w + 2.0 * active * w;
            break;
        case SIB_KERNEL_PROLONG:
            by = 0.75 * n * w + 6.0 * n * w;
            break;
        case SIB_KERNEL_RAS:   // r and x read, xo written (the shared inverse stays on chip)
            by = 9.0 * n * w;
            break;
        case SIB_KERNEL_IB_WINDOW:   // the marker form's words: 15 per marker, 2 per stencil-touched face
            by = (15.0 * c->M + 2.0 * 2.0 * lv.hnRowTiles * lv.tx * lv.ty) * w;
            break;
        default:
            throw SibError(SIB_ERR_ARG, "unknown kernel id");
    }
    if (!cold) launch();   // warm-up
    CK(cudaEventRecord(c->ev0, s));
    for (int r = 0; r < reps; ++r) launch();
    CK(cudaEventRecord(c->ev1, s));
    CK(cudaEventSynchronize(c->ev1));
    kcheck(c);
    float t = 0;
    CK(cudaEventElapsedTime(&t, c->ev0, c->ev1));
    *ms = t / reps;
    *bytes = by;
}

#define API_BEGIN(c)                       \
    if (!(c)) return SIB_ERR_ARG;          \
    try {                                  \
        (c)->err.clear();

#define API_END(c)                                  \
    }                                               \
    catch (const SibError& e) {                     \
        (c)->err = e.what();                        \
        return e.code;                              \
    }                                               \
    catch (const std::exception& e) {               \
        (c)->err = e.what();                        \
        return SIB_ERR_CUDA;                        \
    }

}  // namespace

// ============================================================================================
namespace {
template <typename T>
void cavity_smooth_impl(sib_ctx* c, int l, T* x, const T* b, int sweeps, cudaStream_t s) {
    Level& lv = c->L[l];
    LevelBuf& lb = lv.p[Prec<T>::id];
    const size_t n = (size_t)lv.N * lv.N;
    if (!lb.cav) lb.cav = dalloc(c, sizeof(T) * 5 * n);
    const double om = c->opts.smoother == SIB_SMOOTHER_VANKA ? c->opts.omega : 0.8;
    GridK<T> g = gridk<T>(c, l);
    T* cur = x;
    T* nxt = (T*)lb.xt;
    for (int k = 0; k < sweeps; ++k) {
        ib_apply<T>(c, l, cur, s);
        launch_cavity_vanka<T>(g, cur, b, (T*)lb.r, (T*)lb.cav, nxt, (T)om, s);
        c->launches += 3;
        std::swap(cur, nxt);
    }
    if (cur != x) CK(cudaMemcpyAsync(x, cur, sizeof(T) * 3 * n, cudaMemcpyDeviceToDevice, s));
}

}  // namespace

extern "C" {

void sib_default_opts(sib_opts* o) {
    if (!o) return;
    o->smoother = SIB_SMOOTHER_VANKA;
    o->nu1 = 2;
    o->nu2 = 2;
    o->omega = -1.0;
    o->cheb_iters = 2;
    o->cheb_lo = 0.1;
    o->cheb_hi = 1.1;
    o->power_iters = 10;
    o->vcycle_fp32 = 1;
    o->rtol = 1e-8;
    o->max_it = 100;
    o->restart = 100;
    o->add_SKXn = 1;
    o->use_graphs = 1;
    o->fuse_small = 1;
    o->smooth_krylov = 0;
    o->sc_relax = SIB_RELAX_JACOBI;
    o->box = 4;
    o->box_overlap = 1;
    o->domain = SIB_DOMAIN_PERIODIC;
    o->ras_tc = 1;
    o->l2_persist = 0;
}

static void resolve_opts(sib_opts* o) {
    if (o->omega < 0) o->omega = o->smoother == SIB_SMOOTHER_VANKA ? 0.8 : 1.0;
}

int sib_create(sib_ctx** out, int N, int n_min) {
    if (!out) return SIB_ERR_ARG;
    *out = nullptr;
    if (n_min < 4 || n_min > 16 || (n_min & (n_min - 1)) || N < n_min || N > MAX_N || (N & (N - 1)))
        return SIB_ERR_ARG;
    sib_ctx* c = new (std::nothrow) sib_ctx();
    if (!c) return SIB_ERR_ALLOC;
    try {
        c->N = N;
        c->n_min = n_min;
        int lmax = 0;
        while ((n_min << lmax) < N) ++lmax;
        c->lmax = lmax;
        sib_default_opts(&c->opts);
        resolve_opts(&c->opts);
        c->L.resize(lmax + 1);
        for (int l = 0; l <= lmax; ++l) {
            Level& lv = c->L[l];
            lv.N = n_min << l;
            lv.h = 1.0 / lv.N;
            lv.tx = lv.N < TX ? lv.N : TX;
            lv.ty = lv.N < TY ? lv.N : TY;
            lv.ntx = lv.N / lv.tx;
            lv.nty = lv.N / lv.ty;
            lv.ntiles = lv.ntx * lv.nty;
            lv.W = l == lmax ? 4 : 3;
        }
        {
            int dev = 0;
            CK(cudaGetDevice(&dev));
            CK(cudaDeviceGetAttribute(&c->smemOptin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        }
        CK(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->evFork, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->evJoin, cudaEventDisableTiming));
        for (int l = 1; l <= lmax && l < sib_ctx::LVS; ++l) {
            CK(cudaStreamCreateWithFlags(&c->lvStream[l], cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&c->lvDone[l], cudaEventDisableTiming));
        }
        CK(cudaEventCreate(&c->ev0));
        CK(cudaEventCreate(&c->ev1));
        alloc_level_bufs(c);
        const int N0 = n_min;
        c->n0 = 3 * N0 * N0;
        c->B0 = (double*)dalloc(c, sizeof(double) * 2 * (size_t)N0 * N0 * N0 * N0);
        c->Aug = (double*)dalloc(c, sizeof(double) * 2 * (size_t)c->n0 * c->n0);
        c->Pinv = (double*)dalloc(c, sizeof(double) * (size_t)c->n0 * c->n0);
        c->info = (int*)dalloc(c, sizeof(int));
        c->rasInfo = (int*)dalloc(c, sizeof(int));
        c->piv = (int*)dalloc(c, sizeof(int) * c->n0);
        c->gjWork = dalloc(c, gauss_jordan_work_bytes(c->n0));
        c->flag = (int*)dalloc(c, sizeof(int));
        const size_t n3 = 3 * (size_t)N * N;
        c->rhs = (double*)dalloc(c, sizeof(double) * n3);
        c->zcur = (double*)dalloc(c, sizeof(double) * n3);
        c->fg = (FgDev*)dalloc(c, sizeof(FgDev));
        c->sol = (double*)dalloc(c, sizeof(double) * n3);
        c->res = (double*)dalloc(c, sizeof(double) * n3);
        c->part = (double*)dalloc(c, sizeof(double) * NBLK * 128);
        c->scal = (double*)dalloc(c, sizeof(double) * 512);
        CK(cudaMallocHost(&c->hbuf, sizeof(double) * 512));
        CK(cudaMallocHost(&c->herr, 64));
        std::memset(c->herr, 0, 64);
        alloc_markers(c);
    } catch (const SibError& e) {
        std::fprintf(stderr, "sib_create: %s\n", e.what());
        sib_destroy(c);
        return e.code;
    }
    *out = c;
    return SIB_OK;
}

void sib_destroy(sib_ctx* c) {
    if (!c) return;
    invalidate_graphs(c);
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    if (c->hbuf) cudaFreeHost(c->hbuf);
    if (c->herr) cudaFreeHost(c->herr);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->evFork) cudaEventDestroy(c->evFork);
    if (c->evJoin) cudaEventDestroy(c->evJoin);
    for (int l = 0; l < sib_ctx::LVS; ++l) {
        if (c->lvStream[l]) cudaStreamDestroy(c->lvStream[l]);
        if (c->lvDone[l]) cudaEventDestroy(c->lvDone[l]);
    }
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    delete c;
}

const char* sib_last_error(const sib_ctx* c) { return c ? c->err.c_str() : "null context"; }

int sib_set_fluid(sib_ctx* c, double rho, double mu, double dt) {
    API_BEGIN(c)
    if (!(rho >= 0.0) || !(mu > 0.0) || !(dt > 0.0) || !std::isfinite(rho) || !std::isfinite(mu) || !std::isfinite(dt))
        throw SibError(SIB_ERR_ARG, "need rho >= 0, mu > 0, dt > 0 (finite)");
    c->rho = rho;
    c->mu = mu;
    c->dt = dt;
    c->fluidDirty = true;
    c->kappaDirty = true;   // SC eigen estimates and coarsest operator depend on the fluid too
    invalidate_graphs(c);
    return SIB_OK;
    API_END(c)
}

int sib_set_structure(sib_ctx* c, int M, const double* X, int E, const int32_t* edges, const double* kappa,
                      void* stream) {
    API_BEGIN(c)
    if (M < 0 || E < 0 || (M > 0 && !X) || (E > 0 && (!edges || !kappa)) || (E > 0 && M == 0))
        throw SibError(SIB_ERR_ARG, "invalid structure sizes or null pointers");
    cudaStream_t s = S(stream);
    // validate on the host (set-up time): indices in range, finite positions, kappa >= 0
    std::vector<double> hX(2 * (size_t)M);
    std::vector<int> hE(2 * (size_t)E);
    std::vector<double> hK(E);
    if (M) CK(cudaMemcpyAsync(hX.data(), X, sizeof(double) * 2 * M, cudaMemcpyDeviceToHost, s));
    if (E) {
        CK(cudaMemcpyAsync(hE.data(), edges, sizeof(int) * 2 * E, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(hK.data(), kappa, sizeof(double) * E, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    for (double v : hX) {
        if (!std::isfinite(v)) throw SibError(SIB_ERR_NONFINITE, "marker positions must be finite");
        if (std::fabs(v) > 1e3) throw SibError(SIB_ERR_ARG, "marker positions must lie within 1000 periods");
    }
    for (int v : hE)
        if (v < 0 || v >= M) throw SibError(SIB_ERR_ARG, "edge index out of range");
    for (double v : hK)
        if (!std::isfinite(v) || v < 0.0) throw SibError(SIB_ERR_ARG, "kappa must be finite and >= 0");
    c->M = M;
    c->E = E;
    alloc_markers(c);
    if (M) CK(cudaMemcpyAsync(c->X, X, sizeof(double) * 2 * M, cudaMemcpyDeviceToDevice, s));
    if (E) {
        CK(cudaMemcpyAsync(c->edges, edges, sizeof(int) * 2 * E, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(c->kappa, kappa, sizeof(double) * E, cudaMemcpyDeviceToDevice, s));
    }
    CK(cudaStreamSynchronize(s));
    c->structDirty = true;
    c->kappaDirty = true;
    c->setupDone = false;
    invalidate_graphs(c);
    return SIB_OK;
    API_END(c)
}

int sib_set_stiffness(sib_ctx* c, const double* kappa, void* stream) {
    API_BEGIN(c)
    if (c->E > 0 && !kappa) throw SibError(SIB_ERR_ARG, "null kappa");
    cudaStream_t s = S(stream);
    std::vector<double> hK(c->E);
    if (c->E) {
        CK(cudaMemcpyAsync(hK.data(), kappa, sizeof(double) * c->E, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    for (double v : hK)
        if (!std::isfinite(v) || v < 0.0) throw SibError(SIB_ERR_ARG, "kappa must be finite and >= 0");
    if (c->E) CK(cudaMemcpyAsync(c->kappa, kappa, sizeof(double) * c->E, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    c->kappaDirty = true;
    invalidate_graphs(c);
    return SIB_OK;
    API_END(c)
}

// Widest box subdomain the options accept: up to RAS_EMAX_SMEM cells in shared memory, wider ones
// (boxes of 8 cells with overlap 2, up to RAS_EMAX cells) through the global-workspace set-up and the
// batched correction.
constexpr int RAS_EMAX_ENABLED = RAS_EMAX;
constexpr bool CAVITY_SOLVE_ENABLED = true;

int sib_set_options(sib_ctx* c, const sib_opts* o) {
    API_BEGIN(c)
    if (!o) throw SibError(SIB_ERR_ARG, "null options");
    sib_opts n = *o;
    if ((n.smoother != SIB_SMOOTHER_VANKA && n.smoother != SIB_SMOOTHER_SC && n.smoother != SIB_SMOOTHER_RAS) ||
        n.nu1 < 0 || n.nu2 < 0 || (n.box != 1 && n.box != 2 && n.box != 4 && n.box != 8 && n.box != 16) ||
        n.box_overlap < 0 || (n.box < 16 && n.box + 2 * n.box_overlap > RAS_EMAX_ENABLED) ||
        (n.box == 16 && n.box_overlap > 4) ||
        n.nu1 + n.nu2 > 64 || n.cheb_iters < 1 || n.cheb_iters > 16 || !(n.cheb_lo > 0) || !(n.cheb_hi > n.cheb_lo) ||
        n.power_iters < 1 || n.power_iters > 1000 || !(n.rtol >= 0) || n.max_it < 1 || n.max_it > 100000 ||
        n.restart < 1 || n.restart > 100 || (n.fuse_small != 0 && n.fuse_small != 1) ||
        (n.smooth_krylov != 0 && n.smooth_krylov != 1) || (n.smooth_krylov && (n.nu1 > WRAP_MAXK || n.nu2 > WRAP_MAXK)) ||
        (n.sc_relax != SIB_RELAX_JACOBI && n.sc_relax != SIB_RELAX_SGS) ||
        (n.domain != SIB_DOMAIN_PERIODIC && n.domain != SIB_DOMAIN_CAVITY) || (n.ras_tc != 0 && n.ras_tc != 1) ||
        (n.l2_persist != 0 && n.l2_persist != 1))
        throw SibError(SIB_ERR_ARG, "option out of range");
    if (n.domain == SIB_DOMAIN_CAVITY) {
        if (!CAVITY_SOLVE_ENABLED) throw SibError(SIB_ERR_UNIMPLEMENTED, "the cavity domain is not available");
        if (n.smoother != SIB_SMOOTHER_VANKA || n.smooth_krylov)
            throw SibError(SIB_ERR_UNIMPLEMENTED, "the cavity takes the Vanka smoother with damped sweeps");
    }
    resolve_opts(&n);
    const bool smootherChanged = n.smoother != c->opts.smoother ||
                                 (n.smoother == SIB_SMOOTHER_SC && n.sc_relax != c->opts.sc_relax) ||
                                 (n.smoother == SIB_SMOOTHER_RAS &&
                                  (n.box != c->opts.box || n.box_overlap != c->opts.box_overlap));
    const bool domainChanged = n.domain != c->opts.domain;
    c->opts = n;
    if (n.smooth_krylov) alloc_wrap_bufs(c);
    // the windows (masked in the cavity) and the coarsest operator follow the domain
    if (domainChanged) c->kappaDirty = true;
    // SC needs eigen estimates, RAS its subdomain inverses: both come from sib_setup
    if (smootherChanged && n.smoother != SIB_SMOOTHER_VANKA) c->fluidDirty = true;
    invalidate_graphs(c);
    return SIB_OK;
    API_END(c)
}

int sib_set_eigen_estimates(sib_ctx* c, const double* lamA, const double* lamM) {
    API_BEGIN(c)
    if (!lamA || !lamM) {
        c->lamOverride = false;
    } else {
        c->lamOverride = true;
        c->lamA_ov.assign(lamA, lamA + c->lmax + 1);
        c->lamM_ov.assign(lamM, lamM + c->lmax + 1);
        for (int l = 1; l <= c->lmax; ++l)
            if (!(c->lamA_ov[l] > 0) || !(c->lamM_ov[l] > 0)) throw SibError(SIB_ERR_ARG, "estimates must be > 0");
    }
    c->fluidDirty = true;
    invalidate_graphs(c);
    return SIB_OK;
    API_END(c)
}

int sib_get_eigen_estimates(const sib_ctx* c, double* lamA, double* lamM) {
    if (!c || !lamA || !lamM) return SIB_ERR_ARG;
    for (int l = 0; l <= c->lmax; ++l) {
        lamA[l] = c->L[l].lamA;
        lamM[l] = c->L[l].lamM;
    }
    return SIB_OK;
}

int sib_setup(sib_ctx* c, void* stream) {
    API_BEGIN(c)
    setup(c, S(stream));
    return SIB_OK;
    API_END(c)
}

int sib_solve(sib_ctx* c, const double* g, double* w, sib_stats* st, void* stream) {
    API_BEGIN(c)
    if (!g || !w) throw SibError(SIB_ERR_ARG, "null pointer");
    return solve_impl(c, g, w, st, S(stream), c->opts.add_SKXn != 0);
    API_END(c)
}

int sib_solve_rhs(sib_ctx* c, const double* rhs, double* w, sib_stats* st, void* stream) {
    API_BEGIN(c)
    if (!rhs || !w) throw SibError(SIB_ERR_ARG, "null pointer");
    return solve_impl(c, rhs, w, st, S(stream), false);
    API_END(c)
}

int sib_solve_transpose(sib_ctx* c, const double* rhs, double* w, sib_stats* st, void* stream) {
    API_BEGIN(c)
    if (!rhs || !w) throw SibError(SIB_ERR_ARG, "null pointer");
    // L_IB is symmetric (S = J^T / h^2, K symmetric, -D = G^T), so L^T w = rhs is the forward system
    return solve_impl(c, rhs, w, st, S(stream), false);
    API_END(c)
}

int sib_solve_host(sib_ctx* c, const double* g_host, double* w_host, sib_stats* st, void* stream) {
    API_BEGIN(c)
    if (!g_host || !w_host) throw SibError(SIB_ERR_ARG, "null pointer");
    cudaStream_t s = S(stream);
    const size_t bytes = sizeof(double) * n3f(c);
    CK(cudaMemcpyAsync(c->sol, g_host, bytes, cudaMemcpyHostToDevice, s));
    // solve_impl copies g into its right-hand side before it writes w, so sol can serve as both
    const int rc = solve_impl(c, c->sol, c->sol, st, s, c->opts.add_SKXn != 0);
    CK(cudaMemcpyAsync(w_host, c->sol, bytes, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return rc;
    API_END(c)
}

int sib_grad(sib_ctx* c, const double* w, const double* lam, double* dkappa, double* dX, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    if (!w || !lam || (c->E && !dkappa) || (c->M && !dX)) throw SibError(SIB_ERR_ARG, "null pointer");
    cudaStream_t s = S(stream);
    if (!c->haveIB) {
        if (c->E) CK(cudaMemsetAsync(dkappa, 0, sizeof(double) * c->E, s));
        if (c->M) CK(cudaMemsetAsync(dX, 0, sizeof(double) * 2 * c->M, s));
        return SIB_OK;
    }
    const int M = c->M;
    double* Lam = c->gradTmp;
    double* Y = c->gradTmp + 2 * M;
    double* KY = c->gradTmp + 4 * M;
    double* KLm = c->gradTmp + 6 * M;
    IBK<double> k = ibk<double>(c, c->lmax);
    const double a = c->opts.add_SKXn ? 1.0 : 0.0;
    KL(c, launch_interp<double>(k, w, Y, s));                     // U = J u
    KL(c, launch_axpby<double>(a, c->Xc, c->dt, Y, Y, 2LL * M, s));   // Y = a X + dt U
    KL(c, launch_interp<double>(k, lam, Lam, s));                 // J lam_u
    const double ih2 = (double)c->N * c->N;
    KL(c, launch_axpby<double>(ih2, Lam, 0.0, nullptr, Lam, 2LL * M, s));
    KL(c, launch_spring<double>(c->adjStart, c->adjNbr, c->kap64, M, Y, KY, s));
    KL(c, launch_spring<double>(c->adjStart, c->adjNbr, c->kap64, M, Lam, KLm, s));
    KL(c, launch_grad_kappa(c->edges, c->E, M, Lam, Y, dkappa, s));
    KL(c, launch_grad_X(c->X, M, c->N, w, lam, KY, KLm, c->dt, a, dX, s));
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_num_levels(const sib_ctx* c) { return c ? c->lmax + 1 : SIB_ERR_ARG; }
int sib_level_size(const sib_ctx* c, int l) { return (c && l >= 0 && l <= c->lmax) ? c->L[l].N : SIB_ERR_ARG; }

int sib_apply_operator(sib_ctx* c, int l, int prec, const void* x, void* y, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    check_level(c, l, 0);
    if (!valid_prec(prec) || !x || !y) throw SibError(SIB_ERR_ARG, "bad precision or null pointer");
    if (prec == SIB_PREC_FP64)
        apply_operator<double>(c, l, (const double*)x, nullptr, (double*)y, S(stream));
    else
        apply_operator<float>(c, l, (const float*)x, nullptr, (float*)y, S(stream));
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_cavity_apply_operator(sib_ctx* c, int l, int prec, const void* x, void* y, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    check_level(c, l, 0);
    if (!valid_prec(prec) || !x || !y) throw SibError(SIB_ERR_ARG, "bad precision or null pointer");
    cudaStream_t s = S(stream);
    if (prec == SIB_PREC_FP64) {
        ib_apply<double>(c, l, (const double*)x, s);
        KL(c, launch_cavity_apply<double>(gridk<double>(c, l), (const double*)x, (double*)y, s));
    } else {
        ib_apply<float>(c, l, (const float*)x, s);
        KL(c, launch_cavity_apply<float>(gridk<float>(c, l), (const float*)x, (float*)y, s));
    }
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_cavity_smooth(sib_ctx* c, int l, int prec, void* x, const void* b, int sweeps, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    check_level(c, l, 1);
    if (!valid_prec(prec) || !x || !b || sweeps < 0) throw SibError(SIB_ERR_ARG, "bad argument");
    if (prec == SIB_PREC_FP64)
        cavity_smooth_impl<double>(c, l, (double*)x, (const double*)b, sweeps, S(stream));
    else
        cavity_smooth_impl<float>(c, l, (float*)x, (const float*)b, sweeps, S(stream));
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_apply_ib(sib_ctx* c, int l, int prec, const void* u, void* f, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    check_level(c, l, 0);
    if (!valid_prec(prec) || !u || !f) throw SibError(SIB_ERR_ARG, "bad precision or null pointer");
    cudaStream_t s = S(stream);
    const int64_t nv = 2LL * c->L[l].N * c->L[l].N;
    Level& lv = c->L[l];
    const int pi = prec == SIB_PREC_FP64 ? 0 : 1;
    const size_t es = prec == SIB_PREC_FP64 ? 8 : 4;
    if (pi == 0) {
        ib_apply<double>(c, l, (const double*)u, s);
    } else {
        ib_apply<float>(c, l, (const float*)u, s);
    }
    CK(cudaMemcpyAsync(f, lv.p[pi].fib, es * nv, cudaMemcpyDeviceToDevice, s));
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_smooth(sib_ctx* c, int l, int prec, void* x, const void* b, int sweeps, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    check_level(c, l, 1);
    if (!valid_prec(prec) || !x || !b || sweeps < 0) throw SibError(SIB_ERR_ARG, "bad argument");
    if (prec == SIB_PREC_FP64)
        smooth_impl<double>(c, l, (double*)x, (const double*)b, sweeps, S(stream));
    else
        smooth_impl<float>(c, l, (float*)x, (const float*)b, sweeps, S(stream));
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_residual_restrict(sib_ctx* c, int l, int prec, const void* x, const void* b, void* rc, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    check_level(c, l, 1);
    if (!valid_prec(prec) || !x || !b || !rc) throw SibError(SIB_ERR_ARG, "bad argument");
    cudaStream_t s = S(stream);
    const int Nc = c->L[l - 1].N;
    if (prec == SIB_PREC_FP64) {
        const double* r = (const double*)c->L[l].p[0].r;
        apply_operator<double>(c, l, (const double*)x, (const double*)b, (double*)r, s);
        if (cavity(c))
            KL(c, launch_cavity_restrict<double>(Nc, r, (double*)rc, s));
        else
            KL(c, launch_restrict<double>(Nc, r, (double*)rc, s));
    } else {
        const float* r = (const float*)c->L[l].p[1].r;
        apply_operator<float>(c, l, (const float*)x, (const float*)b, (float*)r, s);
        if (cavity(c))
            KL(c, launch_cavity_restrict<float>(Nc, r, (float*)rc, s));
        else
            KL(c, launch_restrict<float>(Nc, r, (float*)rc, s));
    }
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_prolong_add(sib_ctx* c, int l, int prec, const void* ec, void* xf, void* stream) {
    API_BEGIN(c)
    check_level(c, l, 1);
    if (!valid_prec(prec) || !ec || !xf) throw SibError(SIB_ERR_ARG, "bad argument");
    const int Nc = c->L[l - 1].N;
    if (prec == SIB_PREC_FP64) {
        if (cavity(c))
            KL(c, launch_cavity_prolong_add<double>(Nc, (const double*)ec, (double*)xf, S(stream)));
        else
            KL(c, launch_prolong_add<double>(Nc, (const double*)ec, (double*)xf, S(stream)));
    } else {
        if (cavity(c))
            KL(c, launch_cavity_prolong_add<float>(Nc, (const float*)ec, (float*)xf, S(stream)));
        else
            KL(c, launch_prolong_add<float>(Nc, (const float*)ec, (float*)xf, S(stream)));
    }
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_coarse_solve(sib_ctx* c, int prec, const void* b, void* x, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    if (!valid_prec(prec) || !b || !x) throw SibError(SIB_ERR_ARG, "bad argument");
    if (prec == SIB_PREC_FP64)
        KL(c, launch_coarse_apply<double>(c->Pinv, c->n0, (const double*)b, (double*)x, S(stream)));
    else
        KL(c, launch_coarse_apply<float>(c->Pinv, c->n0, (const float*)b, (float*)x, S(stream)));
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_vcycle(sib_ctx* c, int prec, const void* b, void* z, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    if (!valid_prec(prec) || !b || !z) throw SibError(SIB_ERR_ARG, "bad argument");
    cudaStream_t s = S(stream);
    const int64_t n = n3f(c);
    Level& lv = c->L[c->lmax];
    if (prec == SIB_PREC_FP64) {
        CK(cudaMemcpyAsync(lv.p[0].b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
        double* out = vcycle<double>(c, s);
        CK(cudaMemcpyAsync(z, out, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    } else {
        CK(cudaMemcpyAsync(lv.p[1].b, b, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
        float* out = vcycle<float>(c, s);
        CK(cudaMemcpyAsync(z, out, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    }
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_interp(sib_ctx* c, const double* u, double* U, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    if (!u || (c->M && !U)) throw SibError(SIB_ERR_ARG, "null pointer");
    if (c->M == 0) return SIB_OK;
    cudaStream_t s = S(stream);
    IBK<double> k = ibk<double>(c, c->lmax);
    KL(c, launch_interp<double>(k, u, (double*)c->U[0], s));
    KL(c, launch_interleave((const double*)c->U[0], c->M, U, s));
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_advance_markers(sib_ctx* c, const double* w, double* X_next, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    if (!w || (c->M && !X_next)) throw SibError(SIB_ERR_ARG, "null pointer");
    if (c->M == 0) return SIB_OK;
    cudaStream_t s = S(stream);
    IBK<double> k = ibk<double>(c, c->lmax);
    KL(c, launch_interp<double>(k, w, (double*)c->U[0], s));   // J^n u^{n+1} at the lagged configuration
    KL(c, launch_advance_markers(c->X, (const double*)c->U[0], c->M, c->dt, X_next, s));
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_spread(sib_ctx* c, const double* F, double* f, void* stream) {
    API_BEGIN(c)
    require_setup(c);
    if ((c->M && !F) || !f) throw SibError(SIB_ERR_ARG, "null pointer");
    cudaStream_t s = S(stream);
    const int64_t nv = 2LL * c->N * c->N;
    Level& lv = c->L[c->lmax];
    if (c->M == 0) {
        CK(cudaMemsetAsync(f, 0, sizeof(double) * nv, s));
        return SIB_OK;
    }
    IBK<double> k = ibk<double>(c, c->lmax);
    KL(c, launch_deinterleave(F, c->M, (double*)c->F[0], s));
    CK(cudaMemsetAsync(lv.p[0].fib, 0, sizeof(double) * nv, s));
    KL(c, launch_spread<double>(k, (const double*)c->F[0], (double*)lv.p[0].fib, lv.tiles, lv.nTiles, lv.hnTiles,
                                lv.tx, lv.ty, lv.ntx, lv.spreadWarp, s));
    CK(cudaMemcpyAsync(f, lv.p[0].fib, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
    kcheck(c);
    return SIB_OK;
    API_END(c)
}

int sib_time_kernel(sib_ctx* c, int kernel, int l, int prec, int reps, void* stream, double* ms, double* bytes) {
    API_BEGIN(c)
    const bool cold = (kernel & SIB_TIME_COLD) != 0;
    kernel &= ~SIB_TIME_COLD;
    require_setup(c);
    check_level(c, l, 0);
    if (!valid_prec(prec) || reps < 1 || !ms || !bytes) throw SibError(SIB_ERR_ARG, "bad argument");
    if ((kernel == SIB_KERNEL_RESTRICT || kernel == SIB_KERNEL_PROLONG || kernel == SIB_KERNEL_VANKA ||
         kernel == SIB_KERNEL_RAS || kernel == SIB_KERNEL_RESIDUAL_RESTRICT) && l < 1)
        throw SibError(SIB_ERR_ARG, "kernel needs level >= 1");
    if (kernel == SIB_KERNEL_RAS && c->opts.smoother != SIB_SMOOTHER_RAS)
        throw SibError(SIB_ERR_STATE, "the RAS kernel needs the RAS smoother set up");
    if ((kernel == SIB_KERNEL_SPREAD || kernel == SIB_KERNEL_INTERP || kernel == SIB_KERNEL_IB_WINDOW) && !c->haveIB)
        throw SibError(SIB_ERR_ARG, "no immersed structure");
    if (kernel == SIB_KERNEL_IB_WINDOW && !c->L[l].useWindow)
        throw SibError(SIB_ERR_STATE, "the level has no assembled IB windows");
    if (prec == SIB_PREC_FP64)
        time_kernel<double>(c, kernel, l, reps, cold, S(stream), ms, bytes);
    else
        time_kernel<float>(c, kernel, l, reps, cold, S(stream), ms, bytes);
    return SIB_OK;
    API_END(c)
}

int64_t sib_launch_count(const sib_ctx* c) { return c ? c->launches : 0; }
int64_t sib_device_bytes(const sib_ctx* c) { return c ? c->bytes : 0; }

}  // extern "C"
