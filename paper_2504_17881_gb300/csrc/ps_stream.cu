// Streaming kernels of libps: the single-rotation pair kernel and the FP64
// overlap / norm reductions.  Both read every amplitude once and are bound by
// HBM bandwidth (the reductions of complex64 states by the FP64 pipe).
#include "ps_device.cuh"
#include "ps_internal.h"

namespace ps {

constexpr int kPairThreads = 256;

// Single non-diagonal rotation, complex64: a thread handles two consecutive
// amplitudes j, j+1 (one 16-byte vector, bit h = top bit of x clear in j) and
// their partners j^x, (j+1)^x (one 16-byte vector at (j^x) & ~1, element
// order swapped when x is odd); x == 1 pairs the two halves of one vector.
// Arithmetic identical to the tile kernel: o = cc a + t rotY(b), then o + kdelta * o.
template <bool FULL, bool YODD>
__device__ __forceinline__ void pair_c64_body(float4 *__restrict__ v, int n, uint64_t x, uint64_t z, float base,
                                              float cc, float kdelta) {
    const uint64_t stride = (uint64_t)gridDim.x * kPairThreads;
    const bool do_scale = kdelta != 0.0f;
    auto fin = [&](float2 o) {
        if (do_scale) {
            o.x = fmaf(kdelta, o.x, o.x);
            o.y = fmaf(kdelta, o.y, o.y);
        }
        return o;
    };
    if (x == 1) {
        const uint64_t units = 1ull << (n - 1);
        for (uint64_t u = (uint64_t)blockIdx.x * kPairThreads + threadIdx.x; u < units; u += stride) {
            const uint64_t j = 2 * u;
            const float4 A = v[u];
            const float2 a0 = make_float2(A.x, A.y), a1 = make_float2(A.z, A.w);
            const float t0 = xsign(base, (uint32_t)(__popcll(j & z) & 1) << 31);
            const float2 o0 = fin(rot_update<float, FULL, YODD>(a0, a1, t0, cc));
            const float2 o1 = fin(rot_update<float, FULL, YODD>(a1, a0, YODD ? -t0 : t0, cc));
            v[u] = make_float4(o0.x, o0.y, o1.x, o1.y);
        }
        return;
    }
    const int h = 63 - __clzll(x);
    const uint64_t units = 1ull << (n - 2);
    const uint32_t z0 = (uint32_t)(z & 1) << 31;
    const bool swap = x & 1;
    for (uint64_t u = (uint64_t)blockIdx.x * kPairThreads + threadIdx.x; u < units; u += stride) {
        const uint64_t j = insert_zero(2 * u, h);
        const uint64_t pj = (j ^ x) & ~1ull;
        const float4 A = v[j >> 1];
        const float4 Bv = v[pj >> 1];
        const float2 a0 = make_float2(A.x, A.y), a1 = make_float2(A.z, A.w);
        float2 b0 = make_float2(Bv.x, Bv.y), b1 = make_float2(Bv.z, Bv.w);
        if (swap) {
            const float2 tmp = b0;
            b0 = b1;
            b1 = tmp;
        }
        const uint32_t s0 = (uint32_t)(__popcll(j & z) & 1) << 31;
        const float t0 = xsign(base, s0), t1 = xsign(base, s0 ^ z0);
        const float2 na0 = fin(rot_update<float, FULL, YODD>(a0, b0, t0, cc));
        const float2 na1 = fin(rot_update<float, FULL, YODD>(a1, b1, t1, cc));
        float2 nb0 = fin(rot_update<float, FULL, YODD>(b0, a0, YODD ? -t0 : t0, cc));
        float2 nb1 = fin(rot_update<float, FULL, YODD>(b1, a1, YODD ? -t1 : t1, cc));
        if (swap) {
            const float2 tmp = nb0;
            nb0 = nb1;
            nb1 = tmp;
        }
        v[j >> 1] = make_float4(na0.x, na0.y, na1.x, na1.y);
        v[pj >> 1] = make_float4(nb0.x, nb0.y, nb1.x, nb1.y);
    }
}

__global__ void __launch_bounds__(kPairThreads) k_pair_c64(float2 *__restrict__ psi, int n, const PairParams pp,
                                                           float kdelta) {
    float4 *v = reinterpret_cast<float4 *>(psi);
    const bool full = pp.flags & 2, yodd = pp.flags & 1;
    const float base = (float)pp.base, cc = (float)pp.c;
    if (full) {
        if (yodd) pair_c64_body<true, true>(v, n, pp.x, pp.z, base, cc, kdelta);
        else pair_c64_body<true, false>(v, n, pp.x, pp.z, base, cc, kdelta);
    } else {
        if (yodd) pair_c64_body<false, true>(v, n, pp.x, pp.z, base, 1.0f, kdelta);
        else pair_c64_body<false, false>(v, n, pp.x, pp.z, base, 1.0f, kdelta);
    }
}

// Single non-diagonal rotation, complex128: one 16-byte amplitude and its partner per unit.
template <bool FULL, bool YODD>
__device__ __forceinline__ void pair_c128_body(double2 *__restrict__ psi, int n, uint64_t x, uint64_t z, double base,
                                               double cc, double kdelta) {
    const int h = 63 - __clzll(x);
    const uint64_t units = 1ull << (n - 1);
    const uint64_t stride = (uint64_t)gridDim.x * kPairThreads;
    const bool do_scale = kdelta != 0.0;
    for (uint64_t u = (uint64_t)blockIdx.x * kPairThreads + threadIdx.x; u < units; u += stride) {
        const uint64_t j = insert_zero(u, h);
        const uint64_t pj = j ^ x;
        const double2 a = psi[j], b = psi[pj];
        const double t = xsign(base, (uint32_t)(__popcll(j & z) & 1) << 31);
        double2 na = rot_update<double, FULL, YODD>(a, b, t, cc);
        double2 nb = rot_update<double, FULL, YODD>(b, a, YODD ? -t : t, cc);
        if (do_scale) {
            na.x = fma(kdelta, na.x, na.x);
            na.y = fma(kdelta, na.y, na.y);
            nb.x = fma(kdelta, nb.x, nb.x);
            nb.y = fma(kdelta, nb.y, nb.y);
        }
        psi[j] = na;
        psi[pj] = nb;
    }
}

__global__ void __launch_bounds__(kPairThreads) k_pair_c128(double2 *__restrict__ psi, int n, const PairParams pp,
                                                            double kdelta) {
    const bool full = pp.flags & 2, yodd = pp.flags & 1;
    if (full) {
        if (yodd) pair_c128_body<true, true>(psi, n, pp.x, pp.z, pp.base, pp.c, kdelta);
        else pair_c128_body<true, false>(psi, n, pp.x, pp.z, pp.base, pp.c, kdelta);
    } else {
        if (yodd) pair_c128_body<false, true>(psi, n, pp.x, pp.z, pp.base, 1.0, kdelta);
        else pair_c128_body<false, false>(psi, n, pp.x, pp.z, pp.base, 1.0, kdelta);
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

// Error-free transformations of FP32 values (Dekker's product, Knuth's sum):
// a b = p + e exactly, and acc.hi + v = s + err exactly.  A float pair
// (hi, lo) accumulates a few exact products with about 48 bits of precision;
// it is folded into the FP64 sums every kFoldAmps amplitudes.
struct FloatPair {
    float hi, lo;
};
// The _rn intrinsics keep the compiler from fusing a product into a sum,
// which would break the exactness of both transformations.
__device__ __forceinline__ void pair_add_product(FloatPair &acc, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
}
constexpr int kFoldAmps = 16;

// what = 0: sum |a|^2 ; what = 1: sum conj(a) b.
// complex128: FP64 products and sums.  complex64: each product exact as a
// float pair (its 48 significant bits fit FP64 as well), summed in a float
// pair over kFoldAmps amplitudes, then added to the FP64 sums -- half an FP64
// operation per amplitude instead of four conversions and four FP64 FMAs,
// which left the reduction bound by GB300's FP64 pipe at about 1.1 TB/s.
template <typename R, int WHAT>
__global__ void __launch_bounds__(kReduceThreads) k_reduce1(const typename CT<R>::T *__restrict__ a,
                                                            const typename CT<R>::T *__restrict__ b, uint64_t N,
                                                            double *__restrict__ partials) {
    __shared__ double sh[2 * kReduceThreads / 32];
    double re = 0.0, im = 0.0;
    const uint64_t stride = (uint64_t)gridDim.x * kReduceThreads;
    if constexpr (sizeof(R) == 4) {
        // two amplitudes per 16-byte load (N is even)
        const float4 *a4 = reinterpret_cast<const float4 *>(a);
        const float4 *b4 = reinterpret_cast<const float4 *>(b);
        const uint64_t N2 = N >> 1;
        FloatPair pr{0.f, 0.f}, pi{0.f, 0.f};
        int folded = 0;
        for (uint64_t k = (uint64_t)blockIdx.x * kReduceThreads + threadIdx.x; k < N2; k += stride) {
            const float4 u = a4[k];
            if (WHAT == 0) {
                pair_add_product(pr, u.x, u.x);
                pair_add_product(pr, u.y, u.y);
                pair_add_product(pr, u.z, u.z);
                pair_add_product(pr, u.w, u.w);
            } else {
                const float4 v = b4[k];
                pair_add_product(pr, u.x, v.x);
                pair_add_product(pr, u.y, v.y);
                pair_add_product(pi, u.x, v.y);
                pair_add_product(pi, -u.y, v.x);
                pair_add_product(pr, u.z, v.z);
                pair_add_product(pr, u.w, v.w);
                pair_add_product(pi, u.z, v.w);
                pair_add_product(pi, -u.w, v.z);
            }
            if (++folded == kFoldAmps / 2) {
                re += (double)pr.hi + (double)pr.lo;
                im += (double)pi.hi + (double)pi.lo;
                pr = FloatPair{0.f, 0.f};
                pi = FloatPair{0.f, 0.f};
                folded = 0;
            }
        }
        re += (double)pr.hi + (double)pr.lo;
        im += (double)pi.hi + (double)pi.lo;
    } else {
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

int launch_pair(int dtype, void *psi, int n, const PairParams &pp, double kdelta, void *stream, int num_sms) {
    cudaStream_t st = (cudaStream_t)stream;
    const uint64_t units = 1ull << (n - 1);
    const uint64_t want = (units + kPairThreads - 1) / kPairThreads;
    const uint64_t cap = (uint64_t)num_sms * 8;
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    if (dtype == PS_C64)
        k_pair_c64<<<grid, kPairThreads, 0, st>>>((float2 *)psi, n, pp, (float)kdelta);
    else
        k_pair_c128<<<grid, kPairThreads, 0, st>>>((double2 *)psi, n, pp, kdelta);
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
