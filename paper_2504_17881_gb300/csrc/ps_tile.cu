// Single-window launch of the fused coset-tile pass (see ps_tile.cuh).
#include "ps_tile.cuh"

namespace ps {

template <typename R, int G, int NG>
__global__ void __launch_bounds__(tile_max_threads(sizeof(R), G, NG), 3) k_tile(typename CT<R>::T *__restrict__ psi,
                                                                  const __grid_constant__ TileParams P, int n, R kdelta) {
    tile_pass<R, G, NG, false, true>(psi, psi, P, blockIdx.x, n, kdelta, true, true);
}

// ------------------------------------------------------------------ launch

// Largest register-group count instantiated: 32 complex64 / 16 complex128
// amplitudes per thread at most (0: not instantiated).
template <typename R, int G>
constexpr int ng_max() {
    return ((sizeof(R) == 4 ? 32 : 16) >> G) >= 4 ? 4
           : (((sizeof(R) == 4 ? 32 : 16) >> G) >= 2 ? 2 : (((sizeof(R) == 4 ? 32 : 16) >> G) >= 1 ? 1 : 0));
}

static size_t rec_bytes(int dtype) { return dtype == PS_C64 ? sizeof(KRot<float>) : sizeof(KRot<double>); }

constexpr int kSmemLimit = 200 * 1024;

template <typename R, int G, int NG>
static cudaError_t set_attr_one() {
    if constexpr (NG > ng_max<R, G>()) return cudaSuccess;
    else return cudaFuncSetAttribute(k_tile<R, G, NG>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
}

template <typename R, int G>
static cudaError_t set_tile_attr_all() {
    cudaError_t e = set_attr_one<R, G, 1>();
    if (e == cudaSuccess) e = set_attr_one<R, G, 2>();
    if (e == cudaSuccess) e = set_attr_one<R, G, 4>();
    return e;
}

int prepare_kernels(int dtype) {
    cudaError_t e = cudaSuccess;
    if (dtype == PS_C64) {
        if (e == cudaSuccess) e = set_tile_attr_all<float, 1>();
        if (e == cudaSuccess) e = set_tile_attr_all<float, 2>();
        if (e == cudaSuccess) e = set_tile_attr_all<float, 3>();
        if (e == cudaSuccess) e = set_tile_attr_all<float, 4>();
        if (e == cudaSuccess) e = set_tile_attr_all<float, 5>();
    } else {
        if (e == cudaSuccess) e = set_tile_attr_all<double, 1>();
        if (e == cudaSuccess) e = set_tile_attr_all<double, 2>();
        if (e == cudaSuccess) e = set_tile_attr_all<double, 3>();
        if (e == cudaSuccess) e = set_tile_attr_all<double, 4>();
    }
    return (int)e;
}

// Register groups per thread: the request (0 = 1), capped at 32 complex64 /
// 16 complex128 amplitudes per thread and reduced while a tile would have
// fewer than one warp of threads.
static int groups_per_thread(int dtype, int G, int B, int request) {
    const int amps = dtype == PS_C64 ? 32 : 16;
    int cap = amps >> G;
    cap = cap >= 4 ? 4 : (cap >= 2 ? 2 : 1);
    int ng = request > 0 ? request : 1;
    ng = ng >= 4 ? 4 : (ng >= 2 ? 2 : 1);
    if (ng > cap) ng = cap;
    while (ng > 1 && ((1 << (B - G)) / ng) < 32) ng >>= 1;
    return ng;
}

template <typename R, int G, int NG>
static cudaError_t launch_one(unsigned grid, int threads, size_t bytes, cudaStream_t st, typename CT<R>::T *p,
                              const TileParams &tp, R kdelta) {
    if constexpr (NG > ng_max<R, G>()) {
        return cudaErrorInvalidValue;
    } else {
        k_tile<R, G, NG><<<grid, threads, bytes, st>>>(p, tp, tp.c + tp.d + (31 - __builtin_clz(grid)), kdelta);
        return cudaGetLastError();
    }
}

template <typename R, int G>
static cudaError_t launch_tile_g(int NG, unsigned grid, int threads, size_t bytes, cudaStream_t st,
                                 typename CT<R>::T *p, const TileParams &tp, R kdelta) {
    switch (NG) {
    case 1: return launch_one<R, G, 1>(grid, threads, bytes, st, p, tp, kdelta);
    case 2: return launch_one<R, G, 2>(grid, threads, bytes, st, p, tp, kdelta);
    default: return launch_one<R, G, 4>(grid, threads, bytes, st, p, tp, kdelta);
    }
}

int launch_tile(int dtype, int G, int ng_request, void *psi, int n, const TileParams &tp, double kdelta,
                void *stream, int threads_request) {
    const int B = tp.c + tp.d;
    const size_t bytes = ((size_t)(dtype == PS_C64 ? 8 : 16) << B) + (size_t)tp.nrot * rec_bytes(dtype);
    const unsigned grid = 1u << (n - B);
    const int NG = groups_per_thread(dtype, G, B, ng_request);
    int threads = (1 << (B - G)) / NG;
    const int tmax = tile_max_threads(dtype == PS_C64 ? 4 : 8, G, NG);
    const int cap = (threads_request > 0 && threads_request < tmax) ? threads_request : tmax;
    if (threads > cap) threads = cap;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (dtype == PS_C64) {
        float2 *p = (float2 *)psi;
        const float kd = (float)kdelta;
        switch (G) {
        case 1: e = launch_tile_g<float, 1>(NG, grid, threads, bytes, st, p, tp, kd); break;
        case 2: e = launch_tile_g<float, 2>(NG, grid, threads, bytes, st, p, tp, kd); break;
        case 3: e = launch_tile_g<float, 3>(NG, grid, threads, bytes, st, p, tp, kd); break;
        case 4: e = launch_tile_g<float, 4>(NG, grid, threads, bytes, st, p, tp, kd); break;
        default: e = launch_tile_g<float, 5>(NG, grid, threads, bytes, st, p, tp, kd); break;
        }
    } else {
        double2 *p = (double2 *)psi;
        switch (G) {
        case 1: e = launch_tile_g<double, 1>(NG, grid, threads, bytes, st, p, tp, kdelta); break;
        case 2: e = launch_tile_g<double, 2>(NG, grid, threads, bytes, st, p, tp, kdelta); break;
        case 3: e = launch_tile_g<double, 3>(NG, grid, threads, bytes, st, p, tp, kdelta); break;
        case 4: e = launch_tile_g<double, 4>(NG, grid, threads, bytes, st, p, tp, kdelta); break;
        default: e = cudaErrorInvalidValue; break;
        }
    }
    return (int)e;
}

}  // namespace ps
