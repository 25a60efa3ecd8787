// sm_103a kernels of libps: the fused coset-tile kernel, the pair-streaming
// kernel and the FP64 reductions.  No tensor cores: every kernel streams
// amplitudes and is bound by HBM bandwidth (or, for complex128, by the FP64
// pipe), so the design goal is line-sized, coalesced HBM traffic and few
// instructions per amplitude.
#include <cuda_runtime.h>

#include "ps_internal.h"

namespace ps {

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

__device__ __forceinline__ float flip_sign(float v, uint32_t bit) {
    return __int_as_float(__float_as_int(v) ^ (int)(bit << 31));
}
__device__ __forceinline__ double flip_sign(double v, uint32_t bit) {
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)bit << 63));
}

__device__ __forceinline__ float rot_s(const RotDesc &r, float) { return r.s32; }
__device__ __forceinline__ double rot_s(const RotDesc &r, double) { return r.s64; }
__device__ __forceinline__ float rot_cm1(const RotDesc &r, float) { return r.cm1_32; }
__device__ __forceinline__ double rot_cm1(const RotDesc &r, double) { return r.cm1_64; }

// One rotation on a register group of 2^G amplitudes a[m] (tile index
// j0 ^ U(m)); MU = the rotation's X mask in group coordinates, so a[m]'s
// partner is a[m ^ MU].  Bit m of sbits is the parity of popc(k_m & z) for
// the global index k_m of a[m].  Gather form of cos(phi) I + i sin(phi) P:
//   a'[m] = a[m] + cm1 a[m] + s (-1)^{sbits_m} rotY(a[m ^ MU]).
template <typename R, int G, int MU, int YODD>
__device__ __forceinline__ void rot_group(typename CT<R>::T (&a)[1 << G], R s, R cm1, uint32_t sbits) {
    typename CT<R>::T o[1 << G];
#pragma unroll
    for (int m = 0; m < (1 << G); ++m) {
        const typename CT<R>::T b = a[m ^ MU];
        const R sm = flip_sign(s, (sbits >> m) & 1u);
        const R bx = YODD ? b.x : -b.y;
        const R by = YODD ? b.y : b.x;
        o[m].x = fma(sm, bx, fma(cm1, a[m].x, a[m].x));
        o[m].y = fma(sm, by, fma(cm1, a[m].y, a[m].y));
    }
#pragma unroll
    for (int m = 0; m < (1 << G); ++m) a[m] = o[m];
}

template <typename R, int G, int YODD, int MU>
__device__ __forceinline__ void rot_case(typename CT<R>::T (&a)[1 << G], R s, R cm1, uint32_t sb) {
    if constexpr (MU < (1 << G)) rot_group<R, G, MU, YODD>(a, s, cm1, sb);
}

template <typename R, int G, int YODD>
__device__ __forceinline__ void rot_dispatch(int mu, typename CT<R>::T (&a)[1 << G], R s, R cm1, uint32_t sb) {
    switch (mu) {
    case 0: rot_case<R, G, YODD, 0>(a, s, cm1, sb); break;
    case 1: rot_case<R, G, YODD, 1>(a, s, cm1, sb); break;
    case 2: rot_case<R, G, YODD, 2>(a, s, cm1, sb); break;
    case 3: rot_case<R, G, YODD, 3>(a, s, cm1, sb); break;
    case 4: rot_case<R, G, YODD, 4>(a, s, cm1, sb); break;
    case 5: rot_case<R, G, YODD, 5>(a, s, cm1, sb); break;
    case 6: rot_case<R, G, YODD, 6>(a, s, cm1, sb); break;
    case 7: rot_case<R, G, YODD, 7>(a, s, cm1, sb); break;
    case 8: rot_case<R, G, YODD, 8>(a, s, cm1, sb); break;
    case 9: rot_case<R, G, YODD, 9>(a, s, cm1, sb); break;
    case 10: rot_case<R, G, YODD, 10>(a, s, cm1, sb); break;
    case 11: rot_case<R, G, YODD, 11>(a, s, cm1, sb); break;
    case 12: rot_case<R, G, YODD, 12>(a, s, cm1, sb); break;
    case 13: rot_case<R, G, YODD, 13>(a, s, cm1, sb); break;
    case 14: rot_case<R, G, YODD, 14>(a, s, cm1, sb); break;
    default: rot_case<R, G, YODD, 15>(a, s, cm1, sb); break;
    }
}

__host__ __device__ constexpr int ctz_const(int m) { return (m & 1) ? 0 : 1 + ctz_const(m >> 1); }

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int kTileThreads = 256;

// Fused window: CTA blockIdx.x owns the coset T(k0) of 2^B = 2^(c+d)
// amplitudes (tile index t = seg * 2^c + o  <->  global k0 ^ V(seg) ^ o,
// V(seg) = XOR of v[i] over the set bits i of seg).  Stage it in shared memory
// with 16-byte asynchronous copies, run the register rounds of the window,
// write it back.  Dynamic shared memory: the tile, then the window's RotDescs.
template <typename R, int G>
__global__ void __launch_bounds__(kTileThreads) k_tile(typename CT<R>::T *__restrict__ psi, DevPlanView dp, int wi) {
    using C = typename CT<R>::T;
    constexpr int LS = sizeof(C) == 8 ? 3 : 4;  // log2 bytes per amplitude
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t vtab[4][16];
    const WinDesc *w = dp.win + wi;
    const int c = w->c, d = w->d;
    const int B = c + d;
    const int tid = threadIdx.x;
    C *tile = reinterpret_cast<C *>(smem);
    RotDesc *srot = reinterpret_cast<RotDesc *>(smem + ((size_t)sizeof(C) << B));

    if (tid < 64) {
        const int k = tid >> 4, jj = tid & 15;
        uint64_t acc = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int bi = 4 * k + i;
            if (((jj >> i) & 1) && bi < d) acc ^= w->v[bi];
        }
        vtab[k][jj] = acc;
    }
    {
        // copy this window's rotation descriptors (48-byte records) to shared memory
        const int nwords = w->nrot * (int)(sizeof(RotDesc) / 16);
        const int4 *src = reinterpret_cast<const int4 *>(dp.rot + w->rot_off);
        int4 *dst = reinterpret_cast<int4 *>(srot);
        for (int i = tid; i < nwords; i += blockDim.x) dst[i] = src[i];
    }
    uint64_t k0 = (uint64_t)blockIdx.x << c;
    for (int i = 0; i < d; ++i) {
        const int p = w->piv[i];
        k0 = ((k0 >> p) << (p + 1)) | (k0 & ((1ull << p) - 1));
    }
    __syncthreads();

    const int seg_log = c + LS - 4;  // log2 of 16-byte chunks per segment
    const int nchunks = 1 << (B + LS - 4);
    char *gbase = reinterpret_cast<char *>(psi);
    for (int ch = tid; ch < nchunks; ch += kTileThreads) {
        const uint32_t seg = (uint32_t)ch >> seg_log;
        const uint32_t off = (uint32_t)ch & ((1u << seg_log) - 1);
        const uint64_t V = vtab[0][seg & 15] ^ vtab[1][(seg >> 4) & 15] ^ vtab[2][(seg >> 8) & 15] ^ vtab[3][seg >> 12];
        cp_async16(smem + (size_t)ch * 16, gbase + ((k0 ^ V) << LS) + ((uint64_t)off << 4));
    }
    cp_async_wait_all();
    __syncthreads();

    const int ngroups = 1 << (B - G);
    const int rot_base = w->rot_off;
    for (int si = 0; si < w->nsub; ++si) {
        const SubDesc *sd = dp.sub + w->sub_off + si;
        uint32_t U[1 << G];
        U[0] = 0;
#pragma unroll
        for (int m = 1; m < (1 << G); ++m) U[m] = U[m & (m - 1)] ^ sd->u[ctz_const(m)];
        int piv[G];
#pragma unroll
        for (int i = 0; i < G; ++i) piv[i] = sd->piv[i];
        const int r0 = sd->rot_off - rot_base, r1 = r0 + sd->nrot;
        for (int q = tid; q < ngroups; q += kTileThreads) {
            uint32_t j0 = (uint32_t)q;
#pragma unroll
            for (int i = 0; i < G; ++i) j0 = ((j0 >> piv[i]) << (piv[i] + 1)) | (j0 & ((1u << piv[i]) - 1));
            C a[1 << G];
#pragma unroll
            for (int m = 0; m < (1 << G); ++m) a[m] = tile[j0 ^ U[m]];
            for (int r = r0; r < r1; ++r) {
                const RotDesc &rd = srot[r];
                const uint32_t pb = (__popc(j0 & rd.zt) + __popcll(k0 & rd.z)) & 1u;
                const uint32_t sb = (uint32_t)rd.smask ^ (0u - pb);
                const R s = rot_s(rd, R()), cm1 = rot_cm1(rd, R());
                if (rd.yodd)
                    rot_dispatch<R, G, 1>(rd.mu, a, s, cm1, sb);
                else
                    rot_dispatch<R, G, 0>(rd.mu, a, s, cm1, sb);
            }
#pragma unroll
            for (int m = 0; m < (1 << G); ++m) tile[j0 ^ U[m]] = a[m];
        }
        __syncthreads();
    }

    for (int ch = tid; ch < nchunks; ch += kTileThreads) {
        const uint32_t seg = (uint32_t)ch >> seg_log;
        const uint32_t off = (uint32_t)ch & ((1u << seg_log) - 1);
        const uint64_t V = vtab[0][seg & 15] ^ vtab[1][(seg >> 4) & 15] ^ vtab[2][(seg >> 8) & 15] ^ vtab[3][seg >> 12];
        *reinterpret_cast<int4 *>(gbase + ((k0 ^ V) << LS) + ((uint64_t)off << 4)) =
            *reinterpret_cast<const int4 *>(smem + (size_t)ch * 16);
    }
}

// ------------------------------------------------------------ pair kernel

__device__ __forceinline__ uint64_t insert_zero(uint64_t v, int p) {
    return ((v >> p) << (p + 1)) | (v & ((1ull << p) - 1));
}

template <typename R>
__device__ __forceinline__ typename CT<R>::T pair_update(typename CT<R>::T a, typename CT<R>::T b, R s, R cm1,
                                                         uint32_t sign, uint32_t yodd) {
    const R sm = flip_sign(s, sign);
    const R bx = yodd ? b.x : -b.y;
    const R by = yodd ? b.y : b.x;
    typename CT<R>::T o;
    o.x = fma(sm, bx, fma(cm1, a.x, a.x));
    o.y = fma(sm, by, fma(cm1, a.y, a.y));
    return o;
}

constexpr int kPairThreads = 256;

// Single rotation (x != 0), complex64: a thread handles two consecutive
// amplitudes j, j+1 (one 16-byte vector, bit h = top bit of x clear in j)
// and their partners j^x, (j+1)^x (one 16-byte vector at (j^x) & ~1,
// element order swapped when x is odd).  x == 1 pairs inside one vector.
__global__ void __launch_bounds__(kPairThreads) k_pair_c64(float2 *__restrict__ psi, int n, DevPlanView dp, int wi) {
    const WinDesc *w = dp.win + wi;
    const RotDesc rd = dp.rot[w->rot_off];
    const uint64_t x = rd.x, z = rd.z;
    const float s = rd.s32, cm1 = rd.cm1_32;
    const uint32_t yodd = rd.yodd;
    float4 *v = reinterpret_cast<float4 *>(psi);
    const uint64_t stride = (uint64_t)gridDim.x * kPairThreads;
    if (x == 1) {
        const uint64_t units = 1ull << (n - 1);
        for (uint64_t u = (uint64_t)blockIdx.x * kPairThreads + threadIdx.x; u < units; u += stride) {
            const uint64_t j = 2 * u;
            float4 A = v[u];
            const float2 a0 = make_float2(A.x, A.y), a1 = make_float2(A.z, A.w);
            const uint32_t sg = __popcll(j & z) & 1u;
            const float2 o0 = pair_update<float>(a0, a1, s, cm1, sg, yodd);
            const float2 o1 = pair_update<float>(a1, a0, s, cm1, sg ^ yodd, yodd);
            v[u] = make_float4(o0.x, o0.y, o1.x, o1.y);
        }
        return;
    }
    const int h = 63 - __clzll(x);
    const uint64_t units = 1ull << (n - 2);
    const uint32_t z0 = (uint32_t)(z & 1);
    const bool swap = x & 1;
    for (uint64_t u = (uint64_t)blockIdx.x * kPairThreads + threadIdx.x; u < units; u += stride) {
        const uint64_t j = insert_zero(2 * u, h);
        const uint64_t pj = (j ^ x) & ~1ull;
        const float4 A = v[j >> 1];
        const float4 Bv = v[pj >> 1];
        const float2 a0 = make_float2(A.x, A.y), a1 = make_float2(A.z, A.w);
        float2 b0 = make_float2(Bv.x, Bv.y), b1 = make_float2(Bv.z, Bv.w);
        if (swap) {
            const float2 t = b0;
            b0 = b1;
            b1 = t;
        }
        const uint32_t s0 = __popcll(j & z) & 1u, s1 = s0 ^ z0;
        const float2 na0 = pair_update<float>(a0, b0, s, cm1, s0, yodd);
        const float2 na1 = pair_update<float>(a1, b1, s, cm1, s1, yodd);
        float2 nb0 = pair_update<float>(b0, a0, s, cm1, s0 ^ yodd, yodd);
        float2 nb1 = pair_update<float>(b1, a1, s, cm1, s1 ^ yodd, yodd);
        if (swap) {
            const float2 t = nb0;
            nb0 = nb1;
            nb1 = t;
        }
        v[j >> 1] = make_float4(na0.x, na0.y, na1.x, na1.y);
        v[pj >> 1] = make_float4(nb0.x, nb0.y, nb1.x, nb1.y);
    }
}

// Single rotation (x != 0), complex128: one 16-byte amplitude and its partner per unit.
__global__ void __launch_bounds__(kPairThreads) k_pair_c128(double2 *__restrict__ psi, int n, DevPlanView dp, int wi) {
    const WinDesc *w = dp.win + wi;
    const RotDesc rd = dp.rot[w->rot_off];
    const uint64_t x = rd.x, z = rd.z;
    const double s = rd.s64, cm1 = rd.cm1_64;
    const uint32_t yodd = rd.yodd;
    const int h = 63 - __clzll(x);
    const uint64_t units = 1ull << (n - 1);
    const uint64_t stride = (uint64_t)gridDim.x * kPairThreads;
    for (uint64_t u = (uint64_t)blockIdx.x * kPairThreads + threadIdx.x; u < units; u += stride) {
        const uint64_t j = insert_zero(u, h);
        const uint64_t pj = j ^ x;
        const double2 a = psi[j], b = psi[pj];
        const uint32_t sg = __popcll(j & z) & 1u;
        psi[j] = pair_update<double>(a, b, s, cm1, sg, yodd);
        psi[pj] = pair_update<double>(b, a, s, cm1, sg ^ yodd, yodd);
    }
}

// ------------------------------------------------------------- reductions

constexpr int kReduceBlocks = 1216;  // fixed, so the summation order is fixed
constexpr int kReduceThreads = 256;

template <int NT>
__device__ __forceinline__ void block_sum2(double &re, double &im, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[2 * wid] = re;
        sh[2 * wid + 1] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0, i = 0;
        for (int k = 0; k < NT / 32; ++k) {
            r += sh[2 * k];
            i += sh[2 * k + 1];
        }
        re = r;
        im = i;
    }
}

// what = 0: sum |a|^2 ; what = 1: sum conj(a) b.  FP64 products and sums.
template <typename R, int WHAT>
__global__ void __launch_bounds__(kReduceThreads) k_reduce1(const typename CT<R>::T *__restrict__ a,
                                                            const typename CT<R>::T *__restrict__ b, uint64_t N,
                                                            double *__restrict__ partials) {
    __shared__ double sh[2 * kReduceThreads / 32];
    double re = 0.0, im = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * kReduceThreads;
    for (uint64_t k = (uint64_t)blockIdx.x * kReduceThreads + threadIdx.x; k < N; k += stride) {
        const double ar = (double)a[k].x, ai = (double)a[k].y;
        if (WHAT == 0) {
            re = fma(ar, ar, fma(ai, ai, re));
        } else {
            const double br = (double)b[k].x, bi = (double)b[k].y;
            re = fma(ar, br, fma(ai, bi, re));
            im = fma(ar, bi, fma(-ai, br, im));
        }
    }
    block_sum2<kReduceThreads>(re, im, sh);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = re;
        partials[2 * blockIdx.x + 1] = im;
    }
}

__global__ void __launch_bounds__(kReduceThreads) k_reduce2(const double *__restrict__ partials, int nparts,
                                                            double *__restrict__ out) {
    __shared__ double sh[2 * kReduceThreads / 32];
    double re = 0.0, im = 0.0;
    for (int k = threadIdx.x; k < nparts; k += kReduceThreads) {
        re += partials[2 * k];
        im += partials[2 * k + 1];
    }
    block_sum2<kReduceThreads>(re, im, sh);
    if (threadIdx.x == 0) {
        out[0] = re;
        out[1] = im;
    }
}

// --------------------------------------------------------------- launchers

int reduce_blocks() { return kReduceBlocks; }

template <typename R, int G>
static cudaError_t set_tile_attr(int bytes) {
    return cudaFuncSetAttribute(k_tile<R, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int prepare_kernels(int dtype, int G, int B) {
    const int S = dtype == PS_C64 ? 8 : 16;
    const int bytes = (S << B) + kMaxWindow * (int)sizeof(RotDesc);
    cudaError_t e = cudaSuccess;
    if (dtype == PS_C64) {
        switch (G) {
        case 1: e = set_tile_attr<float, 1>(bytes); break;
        case 2: e = set_tile_attr<float, 2>(bytes); break;
        case 3: e = set_tile_attr<float, 3>(bytes); break;
        default: e = set_tile_attr<float, 4>(bytes); break;
        }
    } else {
        switch (G) {
        case 1: e = set_tile_attr<double, 1>(bytes); break;
        case 2: e = set_tile_attr<double, 2>(bytes); break;
        case 3: e = set_tile_attr<double, 3>(bytes); break;
        default: e = set_tile_attr<double, 4>(bytes); break;
        }
    }
    return (int)e;
}

int launch_tile(int dtype, int G, void *psi, int n, int B, const DevPlanView &dp, const WinDesc &hw, int wi,
                void *stream) {
    const int S = dtype == PS_C64 ? 8 : 16;
    const size_t bytes = ((size_t)S << B) + (size_t)hw.nrot * sizeof(RotDesc);
    const unsigned grid = 1u << (n - B);
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == PS_C64) {
        float2 *p = (float2 *)psi;
        switch (G) {
        case 1: k_tile<float, 1><<<grid, kTileThreads, bytes, st>>>(p, dp, wi); break;
        case 2: k_tile<float, 2><<<grid, kTileThreads, bytes, st>>>(p, dp, wi); break;
        case 3: k_tile<float, 3><<<grid, kTileThreads, bytes, st>>>(p, dp, wi); break;
        default: k_tile<float, 4><<<grid, kTileThreads, bytes, st>>>(p, dp, wi); break;
        }
    } else {
        double2 *p = (double2 *)psi;
        switch (G) {
        case 1: k_tile<double, 1><<<grid, kTileThreads, bytes, st>>>(p, dp, wi); break;
        case 2: k_tile<double, 2><<<grid, kTileThreads, bytes, st>>>(p, dp, wi); break;
        case 3: k_tile<double, 3><<<grid, kTileThreads, bytes, st>>>(p, dp, wi); break;
        default: k_tile<double, 4><<<grid, kTileThreads, bytes, st>>>(p, dp, wi); break;
        }
    }
    return (int)cudaGetLastError();
}

int launch_pair(int dtype, void *psi, int n, const DevPlanView &dp, const WinDesc &hw, int wi, void *stream,
                int num_sms) {
    (void)hw;
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t units = dtype == PS_C64 ? (1ull << (n - 1)) : (1ull << (n - 1));
    uint64_t want = (units + kPairThreads - 1) / kPairThreads;
    uint64_t cap = (uint64_t)num_sms * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    if (dtype == PS_C64)
        k_pair_c64<<<grid, kPairThreads, 0, st>>>((float2 *)psi, n, dp, wi);
    else
        k_pair_c128<<<grid, kPairThreads, 0, st>>>((double2 *)psi, n, dp, wi);
    return (int)cudaGetLastError();
}

int launch_reduce(int dtype, int what, const void *a, const void *b, int n, double *partials, double *out_dev,
                  void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t N = 1ull << n;
    if (dtype == PS_C64) {
        if (what == 0)
            k_reduce1<float, 0><<<kReduceBlocks, kReduceThreads, 0, st>>>((const float2 *)a, nullptr, N, partials);
        else
            k_reduce1<float, 1><<<kReduceBlocks, kReduceThreads, 0, st>>>((const float2 *)a, (const float2 *)b, N,
                                                                          partials);
    } else {
        if (what == 0)
            k_reduce1<double, 0><<<kReduceBlocks, kReduceThreads, 0, st>>>((const double2 *)a, nullptr, N, partials);
        else
            k_reduce1<double, 1><<<kReduceBlocks, kReduceThreads, 0, st>>>((const double2 *)a, (const double2 *)b,
                                                                           N, partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    k_reduce2<<<1, kReduceThreads, 0, st>>>(partials, kReduceBlocks, out_dev);
    return (int)cudaGetLastError();
}

}  // namespace ps
