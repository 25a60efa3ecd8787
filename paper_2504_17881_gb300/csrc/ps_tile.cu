// Fused coset-tile kernel: one HBM pass applies a whole window of rotations.
//
// No tensor cores: the pass streams every amplitude once (read + write) and
// is bound by HBM bandwidth when the on-chip work per amplitude stays small,
// so the kernel is written for few instructions per amplitude and rotation:
// two fused multiply-adds in the tangent form, one sign XOR per pair, and
// per-rotation bookkeeping amortised over all register groups of a thread.
#include "ps_device.cuh"
#include "ps_internal.h"

namespace ps {

// Per-rotation record in shared memory, built by each CTA from RotDesc:
//   coef[i]  signed coefficient of pair base i (or amplitude i when mu == 0):
//            base * (-1)^{parity(U(m) & zt)} for the group index m it stands for;
//   zt       Z mask in tile coordinates;  c  cos(phi) for the full form;
//   meta     bits 0-3 mu, bit 4 popc(x & z) & 1, bit 5 full form,
//            bit 6 parity(k0 & z) of this CTA's coset.
template <typename R> struct KRot;
template <> struct __align__(16) KRot<float> {
    float coef[16];
    uint32_t zt, meta;
    float c, pad;
};
template <> struct __align__(16) KRot<double> {
    double coef[16];
    uint32_t zt, meta;
    double c;
};

// One rotation on the NG register groups of a thread, each of 2^G
// amplitudes a[g][m] (tile index j0_g ^ U(m)).  MU: the rotation's X mask in
// group coordinates (the partner of a[g][m] is a[g][m ^ MU]).  sw[g]: sign
// word (bit 31) of parity(j0_g & zt) ^ parity(k0 & z).  The partner of a
// pair takes the coefficient times (-1)^{popc(x & z)}.
template <typename R, int G, int NG, int MU, int YODD, int FULL>
__device__ __forceinline__ void rot_all(typename CT<R>::T (&a)[NG][1 << G], const KRot<R> &k,
                                        const uint32_t (&sw)[NG]) {
    if constexpr (MU < (1 << G)) {
        using C = typename CT<R>::T;
        constexpr int H = top_bit_const(MU);
        constexpr int NC = MU ? (1 << (G - 1)) : (1 << G);
        R cf[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) cf[i] = k.coef[i];
        const R cc = FULL ? k.c : R(1);
#pragma unroll
        for (int g = 0; g < NG; ++g) {
#pragma unroll
            for (int m = 0; m < (1 << G); ++m) {
                if constexpr (MU == 0) {
                    const R t = xsign(cf[m], sw[g]);
                    a[g][m] = rot_update<R, FULL != 0, false>(a[g][m], a[g][m], t, cc);
                } else if (((m >> H) & 1) == 0) {
                    const int p = m ^ MU;
                    const R t = xsign(cf[pair_index<H>(m)], sw[g]);
                    const C A = a[g][m], Bv = a[g][p];
                    a[g][m] = rot_update<R, FULL != 0, YODD != 0>(A, Bv, t, cc);
                    a[g][p] = rot_update<R, FULL != 0, YODD != 0>(Bv, A, YODD ? -t : t, cc);
                }
            }
        }
    }
}

#define PS_ROT_CASE(k) \
    case k: rot_all<R, G, NG, ((k)&15), (((k) >> 4) & 1), ((k) >> 5)>(a, kr, sw); break;

template <typename R, int G, int NG>
__device__ __forceinline__ void rot_dispatch(int code, typename CT<R>::T (&a)[NG][1 << G], const KRot<R> &kr,
                                             const uint32_t (&sw)[NG]) {
    switch (code) {
        PS_ROT_CASE(0) PS_ROT_CASE(1) PS_ROT_CASE(2) PS_ROT_CASE(3) PS_ROT_CASE(4) PS_ROT_CASE(5)
        PS_ROT_CASE(6) PS_ROT_CASE(7) PS_ROT_CASE(8) PS_ROT_CASE(9) PS_ROT_CASE(10) PS_ROT_CASE(11)
        PS_ROT_CASE(12) PS_ROT_CASE(13) PS_ROT_CASE(14) PS_ROT_CASE(15) PS_ROT_CASE(16) PS_ROT_CASE(17)
        PS_ROT_CASE(18) PS_ROT_CASE(19) PS_ROT_CASE(20) PS_ROT_CASE(21) PS_ROT_CASE(22) PS_ROT_CASE(23)
        PS_ROT_CASE(24) PS_ROT_CASE(25) PS_ROT_CASE(26) PS_ROT_CASE(27) PS_ROT_CASE(28) PS_ROT_CASE(29)
        PS_ROT_CASE(30) PS_ROT_CASE(31) PS_ROT_CASE(32) PS_ROT_CASE(33) PS_ROT_CASE(34) PS_ROT_CASE(35)
        PS_ROT_CASE(36) PS_ROT_CASE(37) PS_ROT_CASE(38) PS_ROT_CASE(39) PS_ROT_CASE(40) PS_ROT_CASE(41)
        PS_ROT_CASE(42) PS_ROT_CASE(43) PS_ROT_CASE(44) PS_ROT_CASE(45) PS_ROT_CASE(46) PS_ROT_CASE(47)
        PS_ROT_CASE(48) PS_ROT_CASE(49) PS_ROT_CASE(50) PS_ROT_CASE(51) PS_ROT_CASE(52) PS_ROT_CASE(53)
        PS_ROT_CASE(54) PS_ROT_CASE(55) PS_ROT_CASE(56) PS_ROT_CASE(57) PS_ROT_CASE(58) PS_ROT_CASE(59)
        PS_ROT_CASE(60) PS_ROT_CASE(61) PS_ROT_CASE(62) PS_ROT_CASE(63)
    default: break;
    }
}
#undef PS_ROT_CASE

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ float base_of(const RotDesc &r, float) { return r.base32; }
__device__ __forceinline__ double base_of(const RotDesc &r, double) { return r.base64; }
__device__ __forceinline__ float cos_of(const RotDesc &r, float) { return r.c32; }
__device__ __forceinline__ double cos_of(const RotDesc &r, double) { return r.c64; }

constexpr int kTileMaxThreads = 256;
constexpr int kVTab = 64;  // entries of the per-iteration segment table

// Fused window: CTA blockIdx.x owns the coset T(k0) of 2^B = 2^(c+d)
// amplitudes (tile index t = seg * 2^c + o  <->  global k0 ^ V(seg) ^ o,
// V(seg) = XOR of v[i] over the set bits i of seg, a linear map).  It stages
// the coset in shared memory with 16-byte asynchronous copies, runs the
// window's register rounds -- each thread owns NG groups of 2^G amplitudes
// and applies the round's rotations to all of them -- multiplies by `scale`
// after the last round, and writes the coset back.  Dynamic shared memory:
// the tile, then the window's rotation records.
template <typename R, int G, int NG>
__global__ void __launch_bounds__(kTileMaxThreads) k_tile(typename CT<R>::T *__restrict__ psi, DevPlanView dp,
                                                          int wi, R scale) {
    using C = typename CT<R>::T;
    constexpr int LS = sizeof(C) == 8 ? 3 : 4;  // log2 bytes per amplitude
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint64_t nib[4][16];  // V over each 4-bit nibble of a segment index
    __shared__ uint64_t vit[kVTab];  // V(i << it_shift) for the load/store iterations
    const WinDesc *w = dp.win + wi;
    const int c = w->c, d = w->d;
    const int B = c + d;
    const int tid = threadIdx.x;
    const int T = blockDim.x;
    const int lgT = 31 - __clz(T);
    C *tile = reinterpret_cast<C *>(smem);
    KRot<R> *srec = reinterpret_cast<KRot<R> *>(smem + ((size_t)sizeof(C) << B));

    uint64_t k0 = (uint64_t)blockIdx.x << c;
    for (int i = 0; i < d; ++i) {
        const int p = w->piv[i];
        k0 = ((k0 >> p) << (p + 1)) | (k0 & ((1ull << p) - 1));
    }
    for (int e = tid; e < 64; e += T) {
        const int k = e >> 4, jj = e & 15;
        uint64_t acc = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int bi = 4 * k + i;
            if (((jj >> i) & 1) && bi < d) acc ^= w->v[bi];
        }
        nib[k][jj] = acc;
    }
    const int nrot = w->nrot;
    for (int e = tid; e < nrot * 16; e += T) {
        const int r = e >> 4, i = e & 15;
        const RotDesc &rd = dp.rot[w->rot_off + r];
        const int mu = rd.mu;
        const int m = mu ? (int)insert_zero((uint64_t)i, 31 - __clz(mu)) : i;
        srec[r].coef[i] = (m < 16) ? xsign(base_of(rd, R()), ((uint32_t)(rd.smask >> m) & 1u) << 31) : R(0);
        if (i == 0) {
            srec[r].zt = rd.zt;
            srec[r].c = cos_of(rd, R());
            srec[r].meta = (uint32_t)mu | ((uint32_t)(rd.flags & 1) << 4) | ((uint32_t)((rd.flags >> 1) & 1) << 5) |
                           ((uint32_t)(__popcll(k0 & rd.z) & 1) << 6);
        }
    }
    __syncthreads();

    // chunk ch = tid + i*T (16 bytes each); when T covers whole segments the
    // segment index splits into disjoint bit fields: tid >> seg_log (low) and
    // i << it_shift (high), so V(seg) = V(low) ^ V(high).
    const int seg_log = c + LS - 4;
    const int nchunks = 1 << (B + LS - 4);
    const int niter = nchunks >> lgT;
    const bool split = lgT >= seg_log;
    const int it_shift = lgT - seg_log;
    auto vof = [&](uint32_t seg) {
        return nib[0][seg & 15] ^ nib[1][(seg >> 4) & 15] ^ nib[2][(seg >> 8) & 15] ^ nib[3][(seg >> 12) & 15];
    };
    if (split) {
        for (int i = tid; i < niter && i < kVTab; i += T) vit[i] = vof((uint32_t)i << it_shift);
        __syncthreads();
    }
    char *gbase = reinterpret_cast<char *>(psi);
    const uint32_t off = (uint32_t)tid & ((1u << seg_log) - 1);
    const uint64_t base = split ? (k0 ^ vof((uint32_t)tid >> seg_log)) : k0;
    auto gaddr = [&](int i) -> uint64_t {
        if (split && i < kVTab) return ((base ^ vit[i]) << LS) + ((uint64_t)off << 4);
        const uint32_t ch = (uint32_t)(tid + (i << lgT));
        return ((k0 ^ vof(ch >> seg_log)) << LS) + ((uint64_t)(ch & ((1u << seg_log) - 1)) << 4);
    };
    for (int i = 0; i < niter; ++i) cp_async16(smem + (size_t)(tid + (i << lgT)) * 16, gbase + gaddr(i));
    cp_async_wait_all();
    __syncthreads();

    const int rot_base = w->rot_off;
    const int nsub = w->nsub;
    const bool do_scale = scale != R(1);
    for (int si = 0; si < nsub; ++si) {
        const SubDesc *sd = dp.sub + w->sub_off + si;
        uint32_t U[1 << G];
        U[0] = 0;
#pragma unroll
        for (int m = 1; m < (1 << G); ++m) U[m] = U[m & (m - 1)] ^ sd->u[ctz_const(m)];
        int piv[G];
#pragma unroll
        for (int i = 0; i < G; ++i) piv[i] = sd->piv[i];
        const int r0 = sd->rot_off - rot_base, r1 = r0 + sd->nrot;
        const bool last = si == nsub - 1;
        const int nbatch = (1 << (B - G)) / (NG * T);
        for (int bt = 0; bt < nbatch; ++bt) {
            uint32_t j0[NG];
#pragma unroll
            for (int g = 0; g < NG; ++g) {
                uint32_t q = (uint32_t)(tid + (bt * NG + g) * T);
#pragma unroll
                for (int i = 0; i < G; ++i) q = ((q >> piv[i]) << (piv[i] + 1)) | (q & ((1u << piv[i]) - 1));
                j0[g] = q;
            }
            C a[NG][1 << G];
#pragma unroll
            for (int g = 0; g < NG; ++g)
#pragma unroll
                for (int m = 0; m < (1 << G); ++m) a[g][m] = tile[j0[g] ^ U[m]];
            for (int r = r0; r < r1; ++r) {
                const KRot<R> &kr = srec[r];
                const uint32_t meta = kr.meta;
                const uint32_t zt = kr.zt;
                const uint32_t tpar = (meta >> 6) & 1u;
                uint32_t sw[NG];
#pragma unroll
                for (int g = 0; g < NG; ++g) sw[g] = ((__popc(j0[g] & zt) ^ tpar) & 1u) << 31;
                rot_dispatch<R, G, NG>((int)(meta & 63u), a, kr, sw);
            }
            if (last && do_scale) {
#pragma unroll
                for (int g = 0; g < NG; ++g)
#pragma unroll
                    for (int m = 0; m < (1 << G); ++m) {
                        a[g][m].x *= scale;
                        a[g][m].y *= scale;
                    }
            }
#pragma unroll
            for (int g = 0; g < NG; ++g)
#pragma unroll
                for (int m = 0; m < (1 << G); ++m) tile[j0[g] ^ U[m]] = a[g][m];
        }
        __syncthreads();
    }

    for (int i = 0; i < niter; ++i)
        *reinterpret_cast<int4 *>(gbase + gaddr(i)) =
            *reinterpret_cast<const int4 *>(smem + (size_t)(tid + (i << lgT)) * 16);
}

// ------------------------------------------------------------------ launch

// Largest register-group count instantiated: 32 complex64 / 16 complex128
// amplitudes per thread at most (more spills).
template <typename R, int G>
constexpr int ng_max() {
    return ((sizeof(R) == 4 ? 32 : 16) >> G) >= 4 ? 4 : (((sizeof(R) == 4 ? 32 : 16) >> G) >= 2 ? 2 : 1);
}

template <typename R, int G, int NG>
static cudaError_t set_tile_attr(int bytes) {
    if constexpr (NG > ng_max<R, G>()) return cudaSuccess;
    else return cudaFuncSetAttribute(k_tile<R, G, NG>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

template <typename R, int G>
static cudaError_t set_tile_attr_all(int bytes) {
    cudaError_t e = set_tile_attr<R, G, 1>(bytes);
    if (e == cudaSuccess) e = set_tile_attr<R, G, 2>(bytes);
    if (e == cudaSuccess) e = set_tile_attr<R, G, 4>(bytes);
    return e;
}

int prepare_kernels(int dtype, int G, int B) {
    const int S = dtype == PS_C64 ? 8 : 16;
    const int bytes = (S << B) + kMaxWindow * (int)(dtype == PS_C64 ? sizeof(KRot<float>) : sizeof(KRot<double>));
    cudaError_t e = cudaSuccess;
    if (dtype == PS_C64) {
        switch (G) {
        case 1: e = set_tile_attr_all<float, 1>(bytes); break;
        case 2: e = set_tile_attr_all<float, 2>(bytes); break;
        case 3: e = set_tile_attr_all<float, 3>(bytes); break;
        default: e = set_tile_attr_all<float, 4>(bytes); break;
        }
    } else {
        switch (G) {
        case 1: e = set_tile_attr_all<double, 1>(bytes); break;
        case 2: e = set_tile_attr_all<double, 2>(bytes); break;
        case 3: e = set_tile_attr_all<double, 3>(bytes); break;
        default: e = set_tile_attr_all<double, 4>(bytes); break;
        }
    }
    return (int)e;
}

// Register groups per thread: the request (0 = 2 for complex64, 1 for
// complex128), capped at 32 complex64 / 16 complex128 amplitudes per thread
// and reduced while a tile would have fewer than one warp of threads.
static int groups_per_thread(int dtype, int G, int B, int request) {
    const int amps = dtype == PS_C64 ? 32 : 16;
    int cap = amps >> G;
    cap = cap >= 4 ? 4 : (cap >= 2 ? 2 : 1);
    int ng = request > 0 ? request : (dtype == PS_C64 ? 2 : 1);
    ng = ng >= 4 ? 4 : (ng >= 2 ? 2 : 1);
    if (ng > cap) ng = cap;
    while (ng > 1 && ((1 << (B - G)) / ng) < 32) ng >>= 1;
    return ng;
}

template <typename R, int G, int NG>
static void launch_one(unsigned grid, int threads, size_t bytes, cudaStream_t st, typename CT<R>::T *p,
                       const DevPlanView &dp, int wi, R scale) {
    if constexpr (NG <= ng_max<R, G>()) k_tile<R, G, NG><<<grid, threads, bytes, st>>>(p, dp, wi, scale);
}

template <typename R, int G>
static void launch_tile_g(int NG, unsigned grid, int threads, size_t bytes, cudaStream_t st, typename CT<R>::T *p,
                          const DevPlanView &dp, int wi, R scale) {
    switch (NG) {
    case 1: launch_one<R, G, 1>(grid, threads, bytes, st, p, dp, wi, scale); break;
    case 2: launch_one<R, G, 2>(grid, threads, bytes, st, p, dp, wi, scale); break;
    default: launch_one<R, G, 4>(grid, threads, bytes, st, p, dp, wi, scale); break;
    }
}

int launch_tile(int dtype, int G, int ng_request, void *psi, int n, int B, const DevPlanView &dp, const WinDesc &hw,
                int wi, double scale, void *stream) {
    const int S = dtype == PS_C64 ? 8 : 16;
    const size_t rec = dtype == PS_C64 ? sizeof(KRot<float>) : sizeof(KRot<double>);
    const size_t bytes = ((size_t)S << B) + (size_t)hw.nrot * rec;
    const unsigned grid = 1u << (n - B);
    const int NG = groups_per_thread(dtype, G, B, ng_request);
    int threads = (1 << (B - G)) / NG;
    if (threads > kTileMaxThreads) threads = kTileMaxThreads;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == PS_C64) {
        float2 *p = (float2 *)psi;
        const float sc = (float)scale;
        switch (G) {
        case 1: launch_tile_g<float, 1>(NG, grid, threads, bytes, st, p, dp, wi, sc); break;
        case 2: launch_tile_g<float, 2>(NG, grid, threads, bytes, st, p, dp, wi, sc); break;
        case 3: launch_tile_g<float, 3>(NG, grid, threads, bytes, st, p, dp, wi, sc); break;
        default: launch_tile_g<float, 4>(NG, grid, threads, bytes, st, p, dp, wi, sc); break;
        }
    } else {
        double2 *p = (double2 *)psi;
        switch (G) {
        case 1: launch_tile_g<double, 1>(NG, grid, threads, bytes, st, p, dp, wi, scale); break;
        case 2: launch_tile_g<double, 2>(NG, grid, threads, bytes, st, p, dp, wi, scale); break;
        case 3: launch_tile_g<double, 3>(NG, grid, threads, bytes, st, p, dp, wi, scale); break;
        default: launch_tile_g<double, 4>(NG, grid, threads, bytes, st, p, dp, wi, scale); break;
        }
    }
    return (int)cudaGetLastError();
}

}  // namespace ps
