// Internal declarations shared by the libps host code and its CUDA kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "ps.h"

namespace ps {

constexpr int kMaxD = 16;       // most basis vectors of one window (tile coordinates above c)
constexpr int kMaxG = 4;        // most group bits in the register stage
constexpr int kMaxWindow = 256; // most rotations per window
constexpr int kMaxN = 40;

// One rotation as the kernels consume it.  `s` carries sin(phi) times
// (-1)^{floor(y/2)} with y = popc(x & z) mod 4, so that the update of
// amplitude j reads (gather form of cos(phi) I + i sin(phi) P):
//   a'[j] = a[j] + cm1 a[j] + s (-1)^{popc(j & z)} rotY(a[j ^ x]),
//   rotY(b) = (-b.im, b.re) for even y, (b.re, b.im) for odd y,
// where cm1 = cos(phi) - 1 = -2 sin^2(phi/2) (no cancellation for small phi).
struct RotDesc {
    double s64, cm1_64;  // FP64 coefficients (PS_C128)
    float s32, cm1_32;   // the same, rounded once to FP32 (PS_C64)
    uint64_t z;          // global Z mask (tile sign)
    uint64_t x;          // global X mask (pair kernel)
    uint32_t zt;         // Z mask in tile coordinates
    uint16_t smask;      // bit m: parity(U(m) & zt), U(m) = combination m of the group basis
    uint8_t mu;          // X mask in group coordinates
    uint8_t yodd;        // popc(x & z) & 1
};

// A register-stage round inside a tile window: every thread owns groups of
// 2^G tile amplitudes {j0 ^ U(m)}, U(m) = XOR of u[i] over the set bits i
// of m, and applies rotations [rot_off, rot_off + nrot) to them in registers.
struct SubDesc {
    uint32_t u[kMaxG];   // group basis in tile coordinates; u[i]'s top bit is piv_of[i]
    int8_t piv[kMaxG];   // pivot positions sorted ascending (coset representatives have zeros there)
    int32_t rot_off;
    int32_t nrot;
};

// One HBM pass.  kind 0 (tile): the 2^n amplitudes split into cosets
// k0 ^ span(v) ^ [0, 2^c) of 2^(c+d) amplitudes each (2^d contiguous
// segments of 2^c); all rotations of the window map every coset to itself.
// kind 1 (pair): a single rotation streamed over the pairs (k, k ^ x).
struct WinDesc {
    uint64_t v[kMaxD];    // basis of V in tile-coordinate order (v[i] <-> tile bit c+i); low c bits zero
    int8_t piv[kMaxD];    // global pivot (top-bit) positions of v, sorted ascending
    int32_t kind;
    int32_t c, d;
    int32_t rot_off, nrot;
    int32_t sub_off, nsub;
    int32_t pad;
};

struct Plan {
    int n = 0;
    int dtype = 0;
    int B = 0;  // tile bits used
    int G = 0;  // group bits used
    std::vector<WinDesc> win;
    std::vector<SubDesc> sub;
    std::vector<RotDesc> rot;
    uint64_t rotations = 0;
};

struct Tuning {
    int B, G, max_window, pair_single, kernel_timing;
};

Tuning resolve_tuning(const ps_tuning *t, int dtype);

// Host scheduler.  Returns PS_OK or PS_ERR_ARG (with message in *err).
int build_plan(int n, int dtype, const uint64_t *x, const uint64_t *z, const double *phi, size_t count,
               const Tuning &tun, Plan &out, std::string *err);

// Host samplers shared by ps_evolve_* and the stream exports.
struct Ham {
    int n;
    std::vector<uint64_t> x, z;
    std::vector<double> h;
};

void set_error(const std::string &msg);

// Kernel launchers (ps_kernels.cu).  Each returns a cudaError_t as int.
struct DevPlanView {
    const WinDesc *win;
    const SubDesc *sub;
    const RotDesc *rot;
};
int launch_tile(int dtype, int G, void *psi, int n, int B, const DevPlanView &dp, const WinDesc &hw, int wi,
                void *stream);
int launch_pair(int dtype, void *psi, int n, const DevPlanView &dp, const WinDesc &hw, int wi, void *stream,
                int num_sms);
int launch_reduce(int dtype, int what, const void *a, const void *b, int n, double *partials, double *out_dev,
                  void *stream);
int reduce_blocks();
int prepare_kernels(int dtype, int G, int B);

}  // namespace ps
