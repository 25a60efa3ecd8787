// Internal declarations shared by the libps host code and its CUDA kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "ps.h"

namespace ps {

constexpr int kMaxD = 16;       // most basis vectors of one window (tile coordinates above c)
constexpr int kMaxG = 5;        // most group bits in the register stage
constexpr int kMaxWindow = 256; // most rotations per window
constexpr int kMaxN = 40;

// One rotation as the kernels consume it.  With y = popc(x & z) mod 4 the
// gather form of exp(i phi P) = cos(phi) I + i sin(phi) P on amplitude j is
//   a'[j] = cos(phi) a[j] + sin(phi) (-1)^{floor(y/2)} (-1)^{popc(j & z)} rotY(a[j ^ x]),
//   rotY(b) = (-b.im, b.re) for even y, (b.re, b.im) for odd y.
// Tangent form (|tan phi| <= 1): a'[j] = cos(phi) (a[j] + base (-1)^{popc(j&z)} rotY(a[j^x]))
// with base = tan(phi) (-1)^{floor(y/2)}; the cos(phi) factors of a window are
// multiplied together and applied once per pass (two fused multiply-adds per
// amplitude and rotation instead of four).  Full form (|tan phi| > 1): base =
// sin(phi) (-1)^{floor(y/2)} and the cos(phi) a[j] term is kept explicitly.
struct RotDesc {
    double base64, c64;  // FP64 coefficients (PS_C128); c64 = cos(phi) for the full form
    float base32, c32;   // the same, rounded once to FP32 (PS_C64)
    uint64_t z;          // global Z mask (coset sign)
    uint64_t x;          // global X mask (pair kernel)
    uint32_t zt;         // Z mask in tile coordinates
    uint32_t smask;      // bit m: parity(U(m) & zt), U(m) = combination m of the group basis
    uint8_t mu;          // X mask in group coordinates
    uint8_t flags;       // bit 0: popc(x & z) & 1; bit 1: full form
};

// A register-stage round inside a tile window: every thread owns groups of
// 2^G tile amplitudes {j0 ^ U(m)}, U(m) = XOR of u[i] over the set bits i
// of m, and applies rotations [rot_off, rot_off + nrot) to them in registers.
// The basis u keeps the rounds' own X masks (so an independent rotation has a
// single-bit group mask); the coset representatives j0 have zeros at the
// pivots of the span's echelon form.
struct SubDesc {
    uint32_t u[kMaxG];   // group basis in tile coordinates
    int8_t piv[kMaxG];   // echelon pivot positions of span(u), sorted ascending
    uint8_t fast;        // k > 0: a standard round of k rotations (see TileSubP::fast)
    int8_t pad[2];
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
    double kprod;         // product of cos(phi) over the window's tangent-form rotations
};

struct Plan {
    int n = 0;
    int dtype = 0;
    int B = 0;  // tile bits used
    int G = 0;  // group bits used
    int NG = 0; // register groups per thread requested (0 = automatic)
    int threads = 0;   // threads per tile-kernel CTA (0: the kernel's default)
    std::vector<WinDesc> win;
    std::vector<SubDesc> sub;
    std::vector<RotDesc> rot;
    uint64_t rotations = 0;
};

struct Tuning {
    int B, G, max_window, pair_single, kernel_timing, reg_groups, seg_bits, tile_threads;
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

// ---------------------------------------------------------------- launches
// Every pass receives its window by value in the kernel's parameter space,
// so a CTA computes its tile addresses and issues its loads without first
// reading descriptors from global memory.

constexpr int kParamRot = 32;  // most rotations of a tile window
constexpr int kParamSub = 16;  // most register rounds of a tile window

struct TileRotP {
    double base;     // signed tan(phi) or sin(phi) (see RotDesc)
    double c;        // cos(phi) for the full form
    uint64_t z;      // global Z mask
    uint32_t zt;     // Z mask in tile coordinates
    uint32_t smask;  // bit m: parity(U(m) & zt)
    uint32_t meta;   // bits 0-4 group X mask mu, bit 5 popc(x & z) & 1, bit 6 full form
    uint32_t pad;
};

// 32 bytes, 16-byte aligned: a pass reads a round's descriptor as two
// 16-byte vectors.
struct alignas(16) TileSubP {
    uint32_t u[kMaxG];  // group basis in tile coordinates
    int8_t piv[kMaxG];  // echelon pivots of span(u), ascending
    uint8_t r0, r1;     // rotations [r0, r1) of the window
    uint8_t fast;       // k > 0: the round is k tangent-form rotations with an even number
                        // of Y factors whose group X masks are 1, 2, 4, ..., 2^(k-1) in order
    uint32_t pad;
};
static_assert(sizeof(TileSubP) == 32 && kMaxG == 5, "round descriptor layout read as two 16-byte vectors");

struct TileParams {
    uint64_t v[kMaxD];  // window basis, v[i] <-> tile bit c + i
    int8_t piv[kMaxD];  // pivots of v, ascending
    int32_t c, d, nsub, nrot;
    TileSubP sub[kParamSub];
    TileRotP rot[kParamRot];
};

struct PairParams {
    uint64_t x, z;
    double base, c;
    uint32_t flags;  // bit 0 popc(x & z) & 1, bit 1 full form
    uint32_t pad;
};

// ------------------------------------------------------------ batched runs
// Many independent runs in one persistent, cooperative launch (ps_batch.cu).

struct BatchRun {
    int32_t n;
    int32_t lane;        // >= 0: lane index; -1: single CTA; -2: single CTA, state resident in shared memory
    uint32_t win_off;    // first window in the batch's window table
    uint32_t nwin;
};

struct BatchWin {
    uint64_t body;       // byte offset of the packed window: head, rounds (padded to 8 bytes), rotations
    double kdelta;       // a <- a + kdelta a after the window's rotations
    int32_t B;           // tile bits c + d
    int16_t nsub, nrot;
};

// Packed window head: the leading part of TileParams (v, piv, c, d, nsub, nrot).
constexpr size_t kWinHeadBytes = offsetof(TileParams, sub);

struct BatchArgs {
    const BatchRun *runs;
    const BatchWin *wins;
    const unsigned char *bodies;
    void *const *states;        // per run: device state (written)
    const void *const *psi0;    // per run: device initial state, or null (evolve the state in place, no overlap)
    double *overlaps;           // per run: re, im
    double *partials;           // two buffers of one (re, im) per lane member
    unsigned *lane_ctr;         // per lane (stride 32 words): arrivals
    unsigned *lane_gen;         // per lane (stride 32 words): barrier generation
    const int *lane_runs;       // runs of each lane, lane by lane
    const int *lane_off;        // nlanes + 1 offsets into lane_runs
    const int *single_order;    // queue order of the single-CTA runs
    unsigned *queue;            // next queue slot
    int *status;                // PS_OK, or PS_ERR_TIMEOUT once a wait ran out
    int nlanes, lane_size, nsingle;
    int withhold;               // test hook: the last member of lane 0 never arrives at a barrier
    long long budget_ns;        // bound of every device-side wait
};

// Resident CTAs per SM of the batched kernel with this dynamic shared memory
// (also raises the kernel's dynamic shared-memory limit to it).
int batch_occupancy(int dtype, size_t smem_bytes, int *blocks_per_sm);
// Cooperative launch of the batched kernel (batch_threads<R>() threads per CTA).
int launch_batch(int dtype, const BatchArgs &a, int grid, size_t smem_bytes, void *stream);
// Bytes of one per-rotation record in a tile pass's shared memory (KRot).
constexpr size_t kRecBytesC64 = 160, kRecBytesC128 = 288;
constexpr int kBatchG = 3;       // group bits of the batched kernel
constexpr int kBatchNG = 2;      // register groups of 2^kBatchG amplitudes per thread
// Most rotations of a batched window.  Every CTA of a batch reserves records
// for this many rotations next to its tile, so three complex128 CTAs of a
// 2^12-amplitude tile (64 KB) fit the SM's 228 KB only with at most 25
// 288-byte records each (24 kept, with room for the static shared memory).
inline int batch_max_window(int dtype) { return dtype == PS_C64 ? kParamRot : 24; }
// Threads per CTA of the batched kernel, sized for three CTAs per SM: 256
// complex64 threads of 16 amplitudes (up to 80 registers each), 128
// complex128 threads of 16 amplitudes (up to 168).  Measured on the 512-run
// workload: 128 complex64 threads of 32 amplitudes were 1.4% slower, and 128
// complex128 threads were 4.6% faster than 256 at 128 registers.
template <typename R>
__host__ __device__ constexpr int batch_threads() { return sizeof(R) == 4 ? 256 : 128; }
constexpr int kLaneStrideWords = 32;

// ------------------------------------------------------ learned step choice
constexpr int kMlpWidth = 128;     // units of each of the three hidden layers
constexpr int kMlpMaxIn = 16;      // most input features
constexpr int kMlpFeatures = 12;   // features of a (Hamiltonian, t, r, initial state) query

struct MlpNorm {
    float mu[kMlpMaxIn], inv_sigma[kMlpMaxIn];
    float y_mu, y_inv_sigma;
};

int mlp_num_params(int n_in);
int mlp_prepare();
int mlp_launch_init(float *P, int n_in, uint64_t seed, void *stream);
int mlp_launch_standardize(const float *x, const float *y, int rows, int n_in, const MlpNorm &nm, float *xs,
                           float *ys, void *stream);
int mlp_launch_forward(const float *P, const float *xs, const int *idx, int rows, int n_in, float *acts, float *out,
                       int denorm, float y_mu, float y_sigma, void *stream);
int mlp_launch_backward(const float *P, const float *ts, const int *idx, int rows, int n_in, float inv_B,
                        const float *acts, const float *out, float *deltas, float *loss_part, void *stream);
int mlp_launch_wgrad(const float *xs, const int *idx, int rows, int n_in, const float *acts, const float *deltas,
                     float *G, void *stream);
int mlp_launch_adam(float *P, const float *G, float *M, float *V, int n, float lr, float beta1, float beta2,
                    float eps, unsigned *count, void *stream);

// A sparse initial state: basis states and their amplitudes.
struct SparseState {
    std::vector<uint64_t> idx;
    std::vector<double> re, im;
};

// Features of "first-order Trotter, r steps to time t from psi" for a
// Hamiltonian whose bound (every term deterministic) is C, whose
// leading-order error coefficient on psi has modulus K_abs and whose
// second-order exponent E2 gives ||E2 psi||^2 = E2_norm2.
void query_features(const Ham &H, double C, double K_abs, double E2_norm2, double t, uint32_t r, float *out);
// The same for a Hamiltonian handle (bound and coefficient cached per state).
int ham_query_features(ps_ham *ham, const uint64_t *idx, const double *amp, size_t ndet, double t, uint32_t r,
                       float *out);

// Kernel parameters of one tile window, from the host copy of a plan.
void fill_tile_params(const Plan &p, const WinDesc &w, TileParams &tp);

// After its rotations a pass applies a <- a + kdelta * a to every amplitude:
// the part of the accumulated cos(phi) factors the state stores.
int launch_tile(int dtype, int G, int ng_request, void *psi, int n, const TileParams &tp, double kdelta,
                void *stream, int threads);
int launch_pair(int dtype, void *psi, int n, const PairParams &pp, double kdelta, void *stream, int num_sms);
int launch_reduce(int dtype, int what, const void *a, const void *b, int n, double *partials, double *out_dev,
                  void *stream);
int reduce_blocks();
int prepare_kernels(int dtype);

}  // namespace ps

// A Hamiltonian handle (include/ps.h): the term list and, once computed,
// its Trotter-error bound with every term deterministic.
struct ps_ham {
    ps::Ham H;
    double bound_full = -1.0;
    // the error coefficient of the last state it was computed for
    ps::SparseState k_state;
    double k_re = 0.0, k_im = 0.0, e2_norm2 = 0.0;
    bool k_valid = false;
};
