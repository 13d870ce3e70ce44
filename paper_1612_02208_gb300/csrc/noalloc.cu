// sib_spread_noalloc: force spreading f = S F on the finest grid for callers that cannot
// allocate device memory.
//
// Some host programs cannot call cudaMalloc at the point where they need a spread: programs
// that have handed the whole device memory to their own pool allocator (a raw cudaMalloc would
// fail or fragment that pool), and latency-critical loops that must not pay for the implicit
// device-wide synchronisation of cudaMalloc/cudaFree.  sib_spread needs a solver context, and
// creating one allocates.  This variant takes only the caller's inputs and output and keeps its
// scratch (marker stencils, the Morton sort, the cell bins and the active-tile list) in one
// file-scope static device array of fixed size, which every GPU that loads the library holds
// until the process exits.
#include <mutex>

#include "sib_internal.h"

namespace {

constexpr int NA_MAX_N = 256;        // grid cells per side
constexpr int NA_MAX_M = 16384;      // markers (a power of two: the sort pads to it)
constexpr int NA_MAX_TILES = (NA_MAX_N / sib::TX) * (NA_MAX_N / sib::TY);

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
// scratch regions, in order
constexpr size_t SZ_BASE = align256(sizeof(int) * NA_MAX_M);                       // x2
constexpr size_t SZ_W64 = align256(sizeof(double) * 8 * NA_MAX_M);                // x2
constexpr size_t SZ_W32 = align256(sizeof(float) * 8 * NA_MAX_M);                 // x2
constexpr size_t SZ_KEYS = align256(sizeof(uint64_t) * NA_MAX_M);
constexpr size_t SZ_SORTED = align256(sizeof(int) * NA_MAX_M);                     // x2
constexpr size_t SZ_MKEY = align256(sizeof(uint32_t) * NA_MAX_M);                  // x2
constexpr size_t SZ_BINS = align256(sizeof(int) * (NA_MAX_N * NA_MAX_N + 1));      // x2
constexpr size_t SZ_FLAG = align256(2 * NA_MAX_TILES);
constexpr size_t SZ_TILES = align256(sizeof(int) * NA_MAX_TILES);
constexpr size_t SZ_NTILES = align256(sizeof(int));
constexpr size_t SZ_F = align256(sizeof(double) * 2 * NA_MAX_M);
constexpr size_t SCRATCH_BYTES = 2 * SZ_BASE + 2 * SZ_W64 + 2 * SZ_W32 + SZ_KEYS + 2 * SZ_SORTED + 2 * SZ_MKEY +
                                 2 * SZ_BINS + SZ_FLAG + SZ_TILES + SZ_NTILES + SZ_F;   // about 4.4 MB

}  // namespace

// The scratch array.  In host code this name is only a host-side stand-in for the device array:
// its device address is obtained with cudaGetSymbolAddress below, on the device that is current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mtx;
unsigned char* g_addr[MAX_DEVICES] = {};

// Device address of the scratch on the current device.  Outside stream capture it is looked up on
// every call (cheap once the module is loaded), so a context re-created after cudaDeviceReset gets
// the array's new address; during capture, where no runtime query should be made, the address of
// the last uncaptured call on this device is used, and a device never called outside capture is an
// error.
int scratch_address(cudaStream_t s, unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return SIB_ERR_CUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return SIB_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mtx);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            g_addr[dev] = nullptr;
            return SIB_ERR_CUDA;
        }
        g_addr[dev] = (unsigned char*)p;
    }
    if (!g_addr[dev]) return SIB_ERR_STATE;
    *out = g_addr[dev];
    return SIB_OK;
}

}  // namespace

extern "C" int sib_spread_noalloc(int N, int M, const double* X, const double* F, double* f, void* stream) {
    using namespace sib;
    if (N < 8 || (N & (N - 1)) || M < 0) return SIB_ERR_ARG;
    if (N > NA_MAX_N || M > NA_MAX_M) return SIB_ERR_TOO_LARGE;
    if (!f || (M > 0 && (!X || !F))) return SIB_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base_addr = nullptr;
    const int rc = scratch_address(s, &base_addr);
    if (rc != SIB_OK) return rc;
    if (cudaMemsetAsync(f, 0, sizeof(double) * 2 * (size_t)N * N, s) != cudaSuccess) return SIB_ERR_CUDA;
    if (M == 0) return cudaGetLastError() == cudaSuccess ? SIB_OK : SIB_ERR_CUDA;

    unsigned char* p = base_addr;
    auto take = [&p](size_t bytes) {
        unsigned char* q = p;
        p += bytes;
        return q;
    };
    int* base[2] = {(int*)take(SZ_BASE), (int*)take(SZ_BASE)};
    double* w64[2] = {(double*)take(SZ_W64), (double*)take(SZ_W64)};
    float* w32[2] = {(float*)take(SZ_W32), (float*)take(SZ_W32)};
    uint64_t* keys = (uint64_t*)take(SZ_KEYS);
    int* sorted[2] = {(int*)take(SZ_SORTED), (int*)take(SZ_SORTED)};
    uint32_t* mkey[2] = {(uint32_t*)take(SZ_MKEY), (uint32_t*)take(SZ_MKEY)};
    int* bins[2] = {(int*)take(SZ_BINS), (int*)take(SZ_BINS)};
    unsigned char* flag = take(SZ_FLAG);
    int* tiles = (int*)take(SZ_TILES);
    int* nTiles = (int*)take(SZ_NTILES);
    double* Fc = (double*)take(SZ_F);

    const int tx = N < TX ? N : TX, ty = N < TY ? N : TY;
    const int ntx = N / tx, nty = N / ty, ntiles = ntx * nty;
    int Mpad = 1;
    while (Mpad < M) Mpad <<= 1;

    // the finest grid is the only level: stencils, Morton order, bins, active tiles
    launch_stencils(X, M, N, 0, base, w64, w32, s);
    launch_deinterleave(F, M, Fc, s);
    for (int q = 0; q < 2; ++q) {
        launch_sort_keys(base[q], M, Mpad, keys, s);
        launch_bitonic(keys, Mpad, s);
        launch_unpack_sorted(keys, M, sorted[q], mkey[q], s);
        launch_bins(mkey[q], M, N * N, 0, bins[q], s);
    }
    // the tile flags must start at zero on every call (the array keeps the last call's contents)
    if (cudaMemsetAsync(flag, 0, 2 * (size_t)ntiles, s) != cudaSuccess) return SIB_ERR_CUDA;
    for (int q = 0; q < 2; ++q) launch_tile_flags(base[q], M, 4, N, tx, ty, ntx, flag, s);
    launch_tile_finish(flag, ntx, nty, tiles, nTiles, s);

    IBK<double> k;
    k.N = N;
    k.W = 4;
    k.M = M;
    k.shift = 0;
    for (int q = 0; q < 2; ++q) {
        k.base[q] = base[q];
        k.wgt[q] = w64[q];
        k.binStart[q] = bins[q];
        k.sorted[q] = sorted[q];
    }
    k.inv_h2 = (double)N * N;
    // one block per tile; blocks past the active-tile count return at once
    launch_spread<double>(k, Fc, f, tiles, nTiles, ntiles, tx, ty, ntx, 0, s);
    return cudaGetLastError() == cudaSuccess ? SIB_OK : SIB_ERR_CUDA;
}
