// Device helpers shared by the libps kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ps {

template <typename R> struct CT;
template <> struct CT<float> { using T = float2; };
template <> struct CT<double> { using T = double2; };

// XOR a sign word (0 or 0x80000000) into the sign bit of v.
__device__ __forceinline__ float xsign(float v, uint32_t sw) { return __int_as_float(__float_as_int(v) ^ (int)sw); }
__device__ __forceinline__ double xsign(double v, uint32_t sw) {
    return __hiloint2double(__double2hiint(v) ^ (int)sw, __double2loint(v));
}

__host__ __device__ constexpr int ctz_const(int m) { return (m & 1) ? 0 : 1 + ctz_const(m >> 1); }
__host__ __device__ constexpr int top_bit_const(int m) { return m <= 1 ? (m == 1 ? 0 : -1) : 1 + top_bit_const(m >> 1); }

// Index of pair base m (bit H clear) among all pair bases of a group, in order.
template <int H>
__host__ __device__ constexpr int pair_index(int m) {
    return H < 0 ? m : ((m & ((1 << H) - 1)) | ((m >> (H + 1)) << H));
}

__device__ __forceinline__ uint64_t insert_zero(uint64_t v, int p) {
    return ((v >> p) << (p + 1)) | (v & ((1ull << p) - 1));
}

// Update of one amplitude a with partner b (gather form, see RotDesc):
//   a' = cc a + t rotY(b),  rotY(b) = (b.x, b.y) for odd y, (-b.y, b.x) for even y,
// cc = cos(phi) in the full form, 1 in the tangent form.
template <typename R, bool FULL, bool YODD>
__device__ __forceinline__ typename CT<R>::T rot_update(typename CT<R>::T a, typename CT<R>::T b, R t, R cc) {
    const R ax = FULL ? cc * a.x : a.x;
    const R ay = FULL ? cc * a.y : a.y;
    typename CT<R>::T o;
    if constexpr (YODD) {
        o.x = fma(t, b.x, ax);
        o.y = fma(t, b.y, ay);
    } else {
        o.x = fma(-t, b.y, ax);
        o.y = fma(t, b.x, ay);
    }
    return o;
}

}  // namespace ps
