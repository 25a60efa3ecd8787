/*
 * ps.h -- C ABI of libps, a single-GPU (GB300, sm_103a) simulator for
 * sequences of Pauli rotations exp(i phi P) applied to a full 2^n complex
 * state vector, the hot path of Miller et al., "phase2: Full-State Vector
 * Simulation of Quantum Time Evolution at Scale" (arXiv:2504.17881).
 *
 * Conventions (all from the paper):
 *   - State: 2^n complex amplitudes, interleaved (re, im), index k = basis
 *     state |k>, qubit q (1-based) = bit q-1, least significant first
 *     (Results, "Software implementation").  PS_C64 stores float pairs
 *     (8 bytes per amplitude), PS_C128 double pairs (16 bytes; the paper's
 *     `_Complex double`, Methods, "Mathematical model").
 *   - Pauli string P = bitmask pair (x, z): bit q of x is set iff factor q+1
 *     is X or Y, bit q of z iff it is Y or Z (Supplementary Methods,
 *     "Pauli-string bit representation"; XIY -> (5, 4)).  Then
 *     P|k> = i^{popc(x&z)} (-1)^{popc(k&z)} |k ^ x>.
 *   - Rotation (x, z, phi) = exp(i phi P) = cos(phi) I + i sin(phi) P
 *     (Results, "Software implementation").  Sequences are given in
 *     application order: element 0 acts first.
 *
 * Memory and streams: the caller owns every state buffer (typically a
 * PyTorch tensor) and the CUDA stream.  The library allocates only its own
 * small device scratch (plan descriptors, reduction partials), freed by the
 * matching destroy call.  Every call that does not return a host value is
 * asynchronous on the state's stream; ps_norm, ps_overlap, ps_get_state and
 * ps_get_stats synchronise that stream.
 *
 * Errors: every int-returning call returns PS_OK or a PS_ERR_* code and
 * leaves a message for ps_last_error() (per host thread).  A call that
 * fails argument validation touches no device memory.  Kernels never trap.
 */
#ifndef PS_H
#define PS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    PS_OK = 0,
    PS_ERR_ARG = 1,         /* invalid argument (null pointer, mask bit >= n, bad size...) */
    PS_ERR_OOM = 2,         /* host or device allocation of library scratch failed */
    PS_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed */
    PS_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out */
    PS_ERR_UNSUPPORTED = 5  /* valid request this build does not support */
};

enum { PS_C64 = 0, PS_C128 = 1 };

/* Kernel kinds reported by ps_get_stats. */
enum { PS_KERNEL_TILE = 0, PS_KERNEL_PAIR = 1, PS_KERNEL_REDUCE = 2, PS_KERNEL_OTHER = 3, PS_KERNEL_KINDS = 4 };

typedef struct ps_state ps_state; /* opaque: one state vector bound to a stream */
typedef struct ps_ham ps_ham;     /* opaque: Hamiltonian term list H = sum_l h_l P_l */
typedef struct ps_plan ps_plan;   /* opaque: a rotation sequence scheduled and resident on the device */

/* Scheduling knobs of the fused path.  Zero in any field selects the default. */
typedef struct ps_tuning {
    int tile_bits;     /* B: log2 amplitudes per fused window tile, 6..13 for PS_C64,
                          6..12 for PS_C128 (default 13 / 12) */
    int group_bits;    /* G: log2 amplitudes per register group, 1..5 for PS_C64, 1..4 for
                          PS_C128 (default 3) */
    int max_window;    /* most rotations per HBM pass (default 64, at most 256) */
    int pair_single;   /* 1: a window holding one non-diagonal rotation runs the pair-streaming
                          kernel instead of the tile kernel; 2: never; 0 = default (1) */
    int kernel_timing; /* 1: time every launch with CUDA events (read with ps_get_stats) */
    int reg_groups;    /* register groups of 2^G amplitudes per thread: 1, 2 or 4 (default 4 for
                          PS_C64, 2 for PS_C128; capped at 32 complex64 / 16 complex128
                          amplitudes per thread) */
    int seg_bits;      /* c_min: log2 of the fewest contiguous amplitudes per segment of a
                          tile, 1..B (default 4 for PS_C64, 3 for PS_C128: 128-byte
                          segments).  A smaller value leaves more tile bits for the window
                          span, so more rotations share a pass, at a finer DRAM access
                          granularity (2^c_min * 8 or 16 bytes). */
    int tile_threads;  /* most threads per CTA of the tile kernel: 64, 128, 256 or 512 (0 =
                          default: 256 while a thread's register groups hold at most 16
                          complex64 / 8 complex128 amplitudes, else 128; a request above that
                          default is capped to it).  Fewer threads give each thread more
                          register batches per round, spreading its fixed per-round work over
                          more amplitudes. */
} ps_tuning;

/* Counters of a state handle since creation or the last ps_reset_stats. */
typedef struct ps_stats {
    uint64_t launches[PS_KERNEL_KINDS];  /* kernel launches per kind */
    double kernel_ms[PS_KERNEL_KINDS];   /* summed CUDA-event time per kind (kernel_timing = 1) */
    double bytes[PS_KERNEL_KINDS];       /* algorithmic HBM bytes per kind (each pass reads and
                                            writes every amplitude once; a reduction reads its inputs) */
    uint64_t rotations;                  /* rotations applied */
    uint64_t passes;                     /* HBM passes (windows) executed */
} ps_stats;

/* Host-side summary of a schedule (no GPU needed to compute it). */
typedef struct ps_plan_info {
    uint64_t rotations;       /* rotations in the sequence */
    uint64_t windows;         /* HBM passes */
    uint64_t tile_windows;    /* passes run by the fused tile kernel */
    uint64_t pair_windows;    /* passes run by the pair-streaming kernel */
    uint64_t subwindows;      /* register-stage rounds summed over tile windows */
    uint64_t fast_subwindows; /* rounds of the standard shape (straight-line code path) */
    uint64_t max_window;      /* longest window (rotations) */
    int tile_bits;            /* B actually used (min(B, n)) */
    int group_bits;           /* G actually used */
} ps_plan_info;

/* ---------------------------------------------------------------- library */

/* Message of the last failing call on this host thread ("" if none). Never NULL. */
const char *ps_last_error(void);

/* ABI version of this header (increments on any signature change). */
int ps_abi_version(void);

/* Number of CUDA devices visible, or -1 if the CUDA driver cannot be loaded. Host only. */
int ps_device_count(void);

/* --------------------------------------------------------------- states */

/* Bind a caller-owned device buffer of 2^n amplitudes (dtype PS_C64 or PS_C128,
 * 16-byte aligned) and a cudaStream_t (NULL = legacy default stream) to a new
 * handle.  1 <= n <= 40.  Does not touch the buffer.  The buffer and stream
 * must outlive the handle. */
int ps_create(int n, int dtype, void *dev_state, void *stream, ps_state **out);

/* Release library scratch owned by the handle (never the caller's buffer).
 * Synchronises the handle's stream first.  NULL is ignored. */
void ps_destroy(ps_state *st);

/* Copy 2^n amplitudes from / to host memory (pinned memory is fastest).
 * ps_set_state is asynchronous: host_src must stay valid until the stream
 * reaches the copy, and it resets the carried scale to 1.  ps_get_state
 * synchronises and returns the STORED amplitudes: the represented state is
 * ps_get_scale() times them (for PS_C64 the factor can differ from 1 by up
 * to 2^-16, more than the complex64 tolerance), so compare with a reference
 * through ps_get_state_represented. */
int ps_set_state(ps_state *st, const void *host_src);
int ps_get_state(ps_state *st, void *host_dst);

/* The state the handle represents, f * (stored amplitudes) with the carried
 * scale f of ps_get_scale, written as 2^n complex128 values (16 bytes per
 * amplitude, re/im interleaved) whatever the handle's dtype.  ps_get_state
 * returns the stored amplitudes, which for PS_C64 differ from the
 * represented state by up to 2^-16 relative; this call applies f in FP64 on
 * the host copy, so a comparison with an FP64 reference needs no extra step.
 * host_dst (caller-owned, 16 * 2^n bytes) is also the staging buffer.
 * Synchronises the state's stream. */
int ps_get_state_represented(ps_state *st, void *host_dst);

/* dst <- src (device to device, on dst's stream); same n and dtype. */
int ps_copy_state(ps_state *dst, const ps_state *src);

/* Scheduling knobs for later calls on this handle (NULL restores defaults). */
int ps_set_tuning(ps_state *st, const ps_tuning *tuning);

/* ------------------------------------------------------------- rotations */

/* psi <- exp(i phi[count-1] P[count-1]) ... exp(i phi[0] P[0]) psi.
 * x, z, phi are host arrays of `count` elements, read before return.  Every
 * mask must have no bit >= n.  count = 0 is a no-op; x = z = 0 applies the
 * global phase exp(i phi).  The sequence is scheduled into HBM passes
 * (windows) on the host -- consecutive rotations whose X masks span a small
 * space share one pass (Eq. 1, common-suffix grouping, in its single-GPU
 * form) -- then the passes are launched on the stream.  Asynchronous. */
int ps_apply_rotations(ps_state *st, const uint64_t *x, const uint64_t *z, const double *phi, size_t count);

/* Schedule a sequence once and keep it on the device: ps_plan_create builds
 * the windows for states of n qubits and `dtype`, uploads them (synchronously,
 * current device) and returns the plan; ps_plan_apply launches it on a state
 * of the same n and dtype (asynchronous, no host work besides the launches).
 * tuning may be NULL (defaults). */
int ps_plan_create(int n, int dtype, const uint64_t *x, const uint64_t *z, const double *phi, size_t count,
                   const ps_tuning *tuning, ps_plan **out);
int ps_plan_apply(ps_state *st, const ps_plan *plan);
int ps_plan_get_info(const ps_plan *plan, ps_plan_info *out);
void ps_plan_destroy(ps_plan *plan);

/* Host only: the summary ps_plan_create would produce, without any GPU. */
int ps_plan_describe(int n, int dtype, const uint64_t *x, const uint64_t *z, const double *phi, size_t count,
                     const ps_tuning *tuning, ps_plan_info *out);

/* Host only: export the schedule for inspection.  For each rotation j:
 * window_of[j] = its window index, and for tile windows its tile-local X and
 * Z masks (xt[j], zt[j]); for each window w: kind[w] (0 tile, 1 pair),
 * c[w] = log2 contiguous amplitudes per segment, d[w] = number of basis
 * vectors and basis[w*16 + i] (i < d[w]) the vectors.  Arrays sized by the
 * caller: count for the per-rotation ones, max_windows for kind, c and d,
 * 16*max_windows for basis.  *n_windows receives the window count (PS_ERR_ARG
 * if it exceeds max_windows). */
int ps_plan_export(int n, int dtype, const uint64_t *x, const uint64_t *z, const double *phi, size_t count,
                   const ps_tuning *tuning, size_t max_windows, size_t *n_windows, uint32_t *window_of,
                   uint32_t *xt, uint32_t *zt, int *kind, int *c, int *d, uint64_t *basis);

/* Stored scale.  A pass applies the cos(phi) factors of its small-angle
 * rotations only to the precision the storage type represents; the residual
 * factor f is tracked in FP64 by the handle, so that the represented state is
 * f * (stored amplitudes).  |f - 1| <= 2^-20 for PS_C128 and 2^-16 for
 * PS_C64 (the factor is applied once it exceeds that, as a <- a + (f - 1) a,
 * so that its rounding is unbiased).  ps_norm and ps_overlap include f; ps_set_state resets it
 * to 1 and ps_copy_state copies it.  This removes the systematic norm drift
 * that per-rotation rounding of cos(phi) ~ 1 to FP32 would cause. */
int ps_get_scale(const ps_state *st, double *out);

/* Measurement helper (no counterpart in the paper): the current device's
 * fused multiply-add throughput in TFLOP/s (2 flops per FMA) for the
 * arithmetic of a dtype -- FP32 for PS_C64, FP64 for PS_C128 -- from
 * independent FMA chains in every thread of a full grid, best of three
 * launches timed with CUDA events (about 0.1 s each).  It is the peak of the
 * ALU roofline of a tile pass whose arithmetic, not HBM, bounds it (the
 * complex128 pass on GB300).  Synchronises the device's default stream. */
int ps_measure_fma_rate(int dtype, double *tflops_out);

/* ------------------------------------------------------------ reductions */

/* *out = <psi|psi> = sum_k |psi[k]|^2, accumulated in FP64 from either dtype
 * in a fixed order (bitwise reproducible on one device).  Synchronises. */
int ps_norm(ps_state *st, double *out);

/* out[0] + i out[1] = <psi0|psi> = sum_k conj(psi0[k]) psi[k] in FP64, the
 * signal g(t) = <psi|exp(i t H)|psi> of Methods, "Data analysis" (Eq. 9)
 * when psi = exp(itH) psi0.  psi0 and psi need the same n and dtype; the
 * work runs on psi's stream and synchronises it. */
int ps_overlap(const ps_state *psi0, ps_state *psi, double out[2]);

/* Allocation-free overlap.  The paper has no counterpart of this call; it is
 * for callers that cannot allocate device memory -- cudaMalloc and cudaFree
 * synchronise the whole device and fail once another allocator (for example
 * a framework's caching allocator, or a budget fixed at start-up) owns the
 * memory, so code that must not stall or that lives inside such a framework
 * has to work with the buffers it already holds.  Unlike ps_overlap it needs
 * no handle (ps_create allocates) and allocates nothing: its partial sums use
 * a fixed device array inside the library (1216 x 2 doubles, about 19 KB,
 * held on every GPU that loads the library until the process exits).
 *
 * Writes <psi0|psi> = sum_k conj(psi0[k]) psi[k] of the stored amplitudes
 * (FP64, same fixed summation order as ps_overlap) as two doubles (re, im) to
 * the caller's device memory out_dev.  psi0_dev, psi_dev: 2^n amplitudes of
 * dtype, 16-byte aligned, on the current device.  Asynchronous on `stream`.
 * n outside [1, 40] (the range the fixed scratch serves) gives PS_ERR_ARG; a
 * current device index of 64 or more gives PS_ERR_UNSUPPORTED (the per-device
 * address cache has 64 entries).
 * The first call on a device looks up the scratch array's device address
 * (one cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the one array: calls that can run at the same
 * time on the GPU (different streams without ordering) race and give wrong
 * results.  Nothing needs clearing between calls. */
int ps_overlap_noalloc(int n, int dtype, const void *psi0_dev, const void *psi_dev, void *stream, double *out_dev);

/* ----------------------------------------------------------- Hamiltonians */

/* Copy a term list H = sum_l h[l] P_l (Eq. 2, Methods, "Hamiltonian
 * simulation") with L >= 1 terms on n qubits; masks must have no bit >= n.
 * Host only. */
int ps_ham_create(int n, size_t L, const uint64_t *x, const uint64_t *z, const double *h, ps_ham **out);
void ps_ham_destroy(ps_ham *ham);

/* lambda = sum_l |h_l|, summed in term order in FP64.  Host only. */
double ps_ham_lambda(const ps_ham *ham);

/* ------------------------------------------------ product-formula streams */
/* Host only.  These write the rotation sequence that the ps_evolve_* calls
 * apply, so callers can inspect, split or batch it. */

/* qDRIFT (Campbell 2019, named in Methods, "Hamiltonian simulation"):
 * draws j = first .. first+count-1 of the N-sample run for `seed`; draw j
 * takes u_j = (SplitMix64 output j+1 of state seed) >> 11, times 2^-53, and
 * selects the smallest l with cdf[l] > u_j * lambda (cdf = running FP64 sum
 * of |h| in term order); it applies exp(i sgn(h_l) (lambda t / N) P_l). */
int ps_qdrift_stream(const ps_ham *ham, double t, uint64_t N, uint64_t seed, uint64_t first, uint64_t count,
                     uint64_t *x_out, uint64_t *z_out, double *phi_out);

/* Number of rotations ps_partial_stream writes: r * (L_D + Ns) (Ns counted
 * only if H_R is non-empty with lambda_R > 0). */
uint64_t ps_partial_length(const ps_ham *ham, size_t L_D, uint32_t r, uint64_t Ns);

/* Partially randomised product formula, first-order reading of Eq. 5
 * (Methods, "Hamiltonian simulation"): H_D = the L_D terms of largest |h|
 * (ties: lower index first), H_R = the rest, both in term order; each of r
 * steps of delta = t / r applies every H_D term as exp(i delta h_l P_l), then
 * Ns draws from H_R as exp(i sgn(h) (lambda_R delta / Ns) P), with one
 * SplitMix64 stream (state seed) running through all steps.  Writes
 * ps_partial_length(...) rotations. */
int ps_partial_stream(const ps_ham *ham, size_t L_D, double t, uint32_t r, uint64_t Ns, uint64_t seed,
                      uint64_t *x_out, uint64_t *z_out, double *phi_out);

/* -------------------------------------------------------- time evolution */

/* First-order Trotter, Eq. 3: (prod_{l=1..L} exp(i (t/r) h_l P_l))^r, term 1
 * applied first in each step.  r >= 1.  Asynchronous. */
int ps_evolve_trotter(ps_state *st, const ps_ham *ham, double t, uint32_t r);

/* qDRIFT with N samples and seed (see ps_qdrift_stream).  Asynchronous. */
int ps_evolve_qdrift(ps_state *st, const ps_ham *ham, double t, uint64_t N, uint64_t seed);

/* Partially randomised formula (see ps_partial_stream).  Asynchronous. */
int ps_evolve_partial(ps_state *st, const ps_ham *ham, size_t L_D, double t, uint32_t r, uint64_t Ns,
                      uint64_t seed);

/* Second order (Methods: the paper's runs use the second-order variant).
 * ps_evolve_trotter2: r symmetric steps of delta = t/r, each applying the
 * terms l = 1..L with angle (delta/2) h_l and then l = L..1 with (delta/2) h_l.
 * The two middle factors of a step and the factors that meet between steps
 * are the same string and are applied as one rotation, so r steps of L
 * terms are r (2L - 2) + 1 rotations (ps_trotter2_length; 1 for L = 1).
 * ps_evolve_partial2: per step, the first L_D terms by decreasing |h|
 * forward with delta/2, then 2 Ns qDRIFT draws from the rest with angle
 * sgn(h) lambda_R delta / (2 Ns), then the same L_D terms backward with
 * delta/2 (the paper fixes only that the randomised part takes twice the
 * samples per step at second order; this symmetric form is the reading
 * used).  It reduces to ps_evolve_trotter2 for L_D = L and to qDRIFT with
 * 2 Ns samples for L_D = 0, r = 1.  Streams as for the first-order calls. */
int ps_evolve_trotter2(ps_state *st, const ps_ham *ham, double t, uint32_t r);
int ps_evolve_partial2(ps_state *st, const ps_ham *ham, size_t L_D, double t, uint32_t r, uint64_t Ns,
                       uint64_t seed);
uint64_t ps_trotter2_length(const ps_ham *ham, uint32_t r);
int ps_trotter2_stream(const ps_ham *ham, double t, uint32_t r, uint64_t *x_out, uint64_t *z_out, double *phi_out);
uint64_t ps_partial2_length(const ps_ham *ham, size_t L_D, uint32_t r, uint64_t Ns);
int ps_partial2_stream(const ps_ham *ham, size_t L_D, double t, uint32_t r, uint64_t Ns, uint64_t seed,
                       uint64_t *x_out, uint64_t *z_out, double *phi_out);
/* Reorder the terms in place by their Pauli strings read from qubit n down
 * to qubit 1, letters I < X < Y < Z, ties in input order (Methods:
 * deterministic terms are ordered lexicographically, so strings that share
 * their upper qubits are applied together). */
int ps_ham_sort_lexicographic(ps_ham *ham);

/* Robust-phase-estimation signal (Methods, "Data analysis"):
 *   Z_m = g(delta 2^m) = <psi0| U(delta)^(2^m) |psi0>,  m = 0..M,
 * U(delta) one step of the order-1 or order-2 product formula (partially
 * randomised when L_D < L and Ns > 0: Ns draws per step at first order,
 * 2 Ns at second).  The state on `work` is continued from round to round,
 * so 2^M steps are applied in total; the draws continue one seed's stream,
 * so Z_m equals a single run of 2^m steps.  Z_out: 2 (M + 1) doubles.
 * Synchronous. */
int ps_rpe_signal(ps_state *work, const ps_state *psi0, const ps_ham *ham, int order, size_t L_D, double delta,
                  uint32_t M, uint64_t Ns, uint64_t seed, double *Z_out);

/* Robust phase estimation of the signal's dominant frequency (Methods,
 * "Data analysis": RPE after Kimmel et al. 2015 recovers the effective
 * ground-state energy from Z_m = g(delta 2^m)).  Z: 2 (M + 1) doubles (re,
 * im of Z_0 .. Z_M), for example from ps_rpe_signal.  With Z_m close to
 * c e^{i 2^m theta}:
 *   theta_0 = arg Z_0 in (-pi, pi];
 *   theta_m = (arg Z_m + 2 pi k) / 2^m, k = floor((2^m theta_{m-1} - arg Z_m) / (2 pi) + 1/2),
 *             the branch nearest theta_{m-1};
 *   *energy_out = theta_M / delta.
 * If every round's phase error |arg Z_m - 2^m theta| (mod 2 pi) is below
 * pi/3, every branch choice is right and theta_M - theta is round M's error
 * divided by 2^M.  The energy is defined modulo 2 pi / delta: callers keep
 * |delta E| < pi (shift H by a multiple of the identity if needed).
 * theta_out (optional, M + 1 doubles) receives every round's estimate.
 * PS_ERR_ARG for M > 62, delta zero or non-finite, or a non-finite Z.
 * Host only. */
int ps_rpe_estimate(const double *Z, uint32_t M, double delta, double *energy_out, double *theta_out);

/* The deterministic size L_D that minimises the cost model of the
 * partially randomised method (Methods, "Hamiltonian simulation"),
 *   C_tot = a L_D / (eps delta) + b lambda_R^2 / eps^2,
 * with the step delta = sqrt(eps / C) set by the analytic bound C(L_D) of
 * ps_ham_trotter_bound (the paper uses a fitted C instead; Methods).
 * L_D runs over 0..L (terms by decreasing |h|); ties keep the smaller L_D.
 * delta_out is +inf when C = 0.  Host only, O(L^2). */
int ps_partial_optimize_split(const ps_ham *ham, double eps, double a, double b, size_t *L_D_out, double *delta_out,
                              double *cost_out);

/* ----------------------------------------------------- sharded schedule
 *
 * A state of n qubits spread over 2^m ranks, as the paper distributes it
 * over nodes (Results, Eq. 1 and its proof in the Supplementary Methods):
 * physical positions 0 .. s-1 (s = n - m) index amplitudes inside a rank's
 * slab of 2^s, positions s .. n-1 are the bits of the rank.  layout[q] is the
 * position of logical qubit q (the identity to start with).
 *
 * ps_shard_swap_plan splits a rotation sequence into steps for rank `rank`:
 *   kind 0, window: rotations [arg_a, arg_b), to be applied to the slab with
 *     the local masks x_out, z_out and the angles phi_out of those indices.
 *     Every X mask of the window is local; Z bits at rank positions only flip
 *     the angle's sign on ranks with odd popc(rank & z_rank) (the +-phi of
 *     Eq. 1 with a diagonal Q).
 *   kind 1, exchange before the next window: swap the rank positions of
 *     mask arg_a with the slab positions of mask arg_b, paired in ascending
 *     order (k = popc(arg_a) pairs: at most k_max, more only when a single
 *     rotation's X mask touches more rank positions).  It is one all-to-all among the
 *     2^k ranks that differ only in the swapped rank bits: ps_shard_pack
 *     orders the slab into 2^k parts (part j goes to the rank whose swapped
 *     bits spell j; the own part stays), and ps_shard_unpack places the part
 *     received from the rank whose swapped bits spell j' -- so every rank
 *     sends and receives (1 - 2^-k) of its slab.
 * A window runs as long as its X masks touch at most k_max rank positions
 * and enough slab qubits stay untouched to swap out; the slab qubits that
 * leave are those whose next use by an X mask lies furthest ahead.  layout
 * is updated to the final layout (pass it to the next call to continue).
 * Arrays: kind, arg_a, arg_b hold up to 2 count entries; x_out, z_out,
 * phi_out count.  Host only.  PS_ERR_ARG for m outside [1, min(n - 1, 20)],
 * k_max outside [1, m], a rank outside [0, 2^m), masks with bits >= n, an X
 * mask on more than n - m qubits (no slab can hold its pairs) or a layout
 * that is not a permutation. */
int ps_shard_swap_plan(int n, int m, int k_max, int rank, const uint64_t *x, const uint64_t *z, const double *phi,
                       size_t count, int32_t *layout, size_t *n_steps, int32_t *kind, uint64_t *arg_a,
                       uint64_t *arg_b, uint64_t *x_out, uint64_t *z_out, double *phi_out);

/* The exchange's data movement on one rank's slab of 2^s amplitudes (dtype
 * PS_C64 / PS_C128, device buffers, distinct, asynchronous on `stream`);
 * lmask: the k slab positions being swapped (1 <= k <= min(20, s)).
 * Packed index i = j 2^(s-k) + c names amplitude c (in the order of the
 * other bits) of part j (the amplitudes whose bits at lmask spell j); the
 * calls move the packed range [first, first + count):
 *   pack:   out[i - first] = slab[the index with the bits of j at lmask and c in the other bits]
 *   unpack: slab[that index] = in[i - first]
 * A whole exchange packs part j for the rank whose swapped bits spell j and
 * unpacks, at part j', what the rank whose swapped bits spell j' sent; done
 * part by part (the own part stays), or in chunks of a part, a rank needs two
 * chunk buffers beside its slab.  PS_ERR_ARG for a range outside 2^s. */
int ps_shard_pack(int s, int dtype, uint64_t lmask, uint64_t first, uint64_t count, const void *slab_dev,
                  void *out_dev, void *stream);
int ps_shard_unpack(int s, int dtype, uint64_t lmask, uint64_t first, uint64_t count, const void *in_dev,
                    void *slab_dev, void *stream);

/* ------------------------------------------------------------ statistics */

/* Counters since creation or the last reset; synchronises the stream when
 * kernel timing is on. */
int ps_get_stats(ps_state *st, ps_stats *out);
int ps_reset_stats(ps_state *st);

/* --------------------------------------------------------------- batches
 *
 * Many independent runs in one persistent launch.  The paper runs its
 * independent simulations -- other Hamiltonians, times, step counts and
 * random samples -- as separate jobs, hundreds at a time (Methods,
 * "Computational details"); here they share one cooperative kernel,
 * replayed from a CUDA graph:
 *   - runs with n <= resident_bits keep their whole state in one CTA's
 *     shared memory for all their windows;
 *   - other runs with n <= single_bits run on one CTA, tile by tile;
 *   - larger runs go to lanes of lane_size co-resident CTAs that split each
 *     window's tiles and meet at a bounded-wait barrier before the next;
 *   - lanes get their runs longest first (work 2^n x windows) on the host,
 *     and every CTA that has finished its lane takes single runs from a
 *     device queue, longest first.
 * Every run starts from psi0 (read-only; the state is written by the first
 * window), so a replay recomputes the same result, and ends with the FP64
 * overlap <psi0|psi> summed in a fixed order.  The evolved state is stored
 * exactly (no pending cos(phi) scale: the last window applies all of it).
 * A device-side wait that runs out (wait_ms) makes the launch return
 * PS_ERR_TIMEOUT from ps_batch_wait; the states are then undefined.
 */
typedef struct ps_batch ps_batch; /* opaque: scheduled runs resident on one device */

typedef struct ps_run_desc {
    int n;             /* qubits, 4..30 */
    void *state;       /* device buffer of 2^n amplitudes of the batch dtype, 16-byte aligned; receives
                          the evolved state.  Runs never share a state buffer. */
    const void *psi0;  /* device initial state (read only; runs may share one), or NULL: the run evolves
                          `state` in place, a replay continues from where the last one ended, and the
                          overlap reported is 0 */
    const uint64_t *x; /* host arrays of `count` rotations in application order, copied at creation */
    const uint64_t *z;
    const double *phi;
    size_t count;
} ps_run_desc;

/* Zero in any field selects the default. */
typedef struct ps_batch_config {
    int lane_size;     /* CTAs per lane: a power of two, 1..256 (default 16) */
    int tile_bits;     /* largest tile of a lane or single run, 8..13 for PS_C64 and 8..12 for PS_C128
                          (default 13 / 12); a lane run of n qubits uses
                          min(tile_bits, max(8, n - log2(lane_size))) */
    int resident_bits; /* runs with n <= resident_bits are resident in shared memory; at most 13 (PS_C64)
                          / 12 (PS_C128), the default; -1: none */
    int single_bits;   /* runs with n <= single_bits (and not resident) run on one CTA; -1: none;
                          default resident_bits + 1 */
    int use_graph;     /* default / 1: capture the launch in a CUDA graph; -1: plain launches */
    int wait_ms;       /* bound of every device-side wait, milliseconds (default 5000) */
    int test_withhold; /* test hook: 1 makes the last CTA of lane 0 skip its barrier arrivals, so the
                          lane's waits run out and ps_batch_wait returns PS_ERR_TIMEOUT */
} ps_batch_config;

typedef struct ps_batch_info {
    uint64_t runs, lane_runs, single_runs, resident_runs;
    uint64_t rotations;         /* summed over runs */
    uint64_t windows;           /* tile passes summed over runs */
    double amplitude_passes;    /* sum over runs of 2^n x windows */
    double amplitude_rotations; /* sum over runs of 2^n x rotations */
    uint64_t body_bytes;        /* device bytes of the packed windows */
    uint64_t smem_bytes;        /* dynamic shared memory per CTA */
    double max_lane_work;       /* largest lane's sum of 2^n x (windows + 1) */
    double single_work;         /* the same summed over single runs */
    int grid, ctas_per_sm, lanes, lane_size, tile_bits, resident_bits, single_bits, graph;
} ps_batch_info;

/* Schedule every run (host, in parallel threads), upload the windows and
 * prepare the launch on `stream` (a cudaStream_t; the current device).
 * A batched window holds at most 32 (PS_C64) or 24 (PS_C128) rotations, so
 * that three CTAs with their tiles and per-rotation records share an SM.
 * Fails with PS_ERR_ARG on an invalid run (n outside 4..30, null or
 * misaligned buffers, a state shared by two runs or aliasing a psi0, a mask
 * bit >= n, a non-finite angle) or configuration, PS_ERR_OOM when device
 * memory runs out, PS_ERR_CUDA when the cooperative launch cannot hold the
 * grid. */
int ps_batch_create(int dtype, const ps_run_desc *runs, size_t nruns, const ps_batch_config *cfg, void *stream,
                    ps_batch **out);
/* Start all runs (asynchronous on the batch's stream). */
int ps_batch_launch(ps_batch *b);
/* Wait for the last launch; copy 2*nruns doubles (re, im of <psi0|psi> per
 * run) to `overlaps` unless it is NULL.  PS_ERR_TIMEOUT if a wait ran out. */
int ps_batch_wait(ps_batch *b, double *overlaps);
/* ps_batch_launch then ps_batch_wait. */
int ps_batch_run(ps_batch *b, double *overlaps);
int ps_batch_get_info(const ps_batch *b, ps_batch_info *out);
void ps_batch_destroy(ps_batch *b);

/* Host-only dry run of ps_batch_create for an assumed grid (ctas_per_sm x
 * num_sms CTAs): the schedule without device work.  state and psi0 may be
 * NULL.  Per run, lane_of receives the lane (>= 0), -1 (single CTA) or -2
 * (resident), tile_bits_of the tile bits and windows_of the windows; any of
 * the three may be NULL. */
int ps_batch_describe(int dtype, const ps_run_desc *runs, size_t nruns, const ps_batch_config *cfg, int num_sms,
                      int ctas_per_sm, ps_batch_info *out, int *lane_of, int *tile_bits_of, uint64_t *windows_of);

/* --------------------------------------------------- learned step choice
 *
 * The paper's error target (eps = 0.001, Methods, "Hamiltonian simulation")
 * fixes the Trotter step count r through the error prefactor, whose analytic
 * bound (Methods, "Data analysis") it finds one to two orders of magnitude
 * too large (Results).  Here a small network predicts the natural log of the
 * empirical first-order Trotter error of the overlap,
 *     eps(H, t, r) = |<psi|U_r(t)|psi> - <psi|exp(itH)|psi>|,
 * from ten features of the query, trained on errors the simulator itself
 * produces; r is then the smallest step count whose prediction is at most
 * log(eps) - margin.  The plain doubling sweep (ps_trotter_sweep) is the
 * fallback and the judge.
 */
#define PS_MLP_FEATURES 12

/* The bound on the Trotter-error prefactor of the partially randomised
 * decomposition with deterministic part D = the first L_D terms by
 * decreasing |h| (ties in input order) and randomised one-norm lambda_R:
 *   4 sum_{l in D} |h_l| sum_{k in D, P_k anticommutes with P_l} |h_k|
 *     + lambda_R (lambda - lambda_R)^2 + (lambda - lambda_R) lambda_R^2
 * (Methods, "Data analysis").  Host only, O(L_D^2). */
int ps_ham_trotter_bound(const ps_ham *ham, size_t L_D, double *out);

/* The step count the analytic bound gives for first-order Trotter (every
 * term deterministic): the paper's error model eps = C delta^2 with
 * delta = t / r (Methods, "Hamiltonian simulation"), so
 * r = max(1, ceil(t sqrt(C / eps))), C = ps_ham_trotter_bound(ham, L).
 * PS_ERR_ARG for t or eps not positive; PS_ERR_UNSUPPORTED when r would
 * exceed 2^32 - 1.  Host only. */
int ps_ham_bound_steps(const ps_ham *ham, double t, double eps, uint32_t *r_out);

/* Three-point Richardson extrapolation to r -> infinity of first-order
 * product-formula overlaps g_r = g + a / r + b / r^2 + O(r^-3) (Eq. 3 has a
 * first-order error): out = (8 g_4R - 6 g_2R + g_R) / 3 from runs at R, 2R,
 * 4R.  Complex values as (re, im).  Host only. */
int ps_richardson3(const double g_R[2], const double g_2R[2], const double g_4R[2], double out[2]);

/* Training labels of the learned step choice: for each of `count` overlaps
 * g (re, im pairs), eps_out[i] = |g_i - g_lim| and
 * log_eps_out[i] = log(max(eps_out[i], eps_floor)) (eps_floor > 0).
 * Host only. */
int ps_trotter_error_labels(const double *g, size_t count, const double g_lim[2], double eps_floor, double *eps_out,
                            float *log_eps_out);

/* The pick margin: the `quantile` (0..1) of the held-out residuals
 * y[i] - pred[i] (log error minus prediction, in FP64), at least 0, so that
 * prediction + margin bounds the error in about that fraction of cases.
 * The quantile interpolates linearly between the sorted residuals at
 * position quantile * (count - 1).  Host only. */
int ps_mlp_margin(const float *y, const float *pred, size_t count, double quantile, double *margin_out);

/* The leading coefficient K of the first-order Trotter error of the overlap
 * for the sparse initial state psi = sum_i amp_i |idx_i> (ndet distinct
 * basis states; amp holds re, im pairs):
 *   K = sum_{k < l, P_k P_l = -P_l P_k} h_l h_k <psi|P_l P_k|psi>,
 * term k applied before term l.  One Trotter step of size delta equals
 * exp(i delta H - (delta^2 / 2) sum_{l>k} h_l h_k [P_l, P_k] + O(delta^3)),
 * so g_r(t) - g(t) = -(t^2 / r) K + O(t^3 / r).  out = (re of K, im of K,
 * ||E2 psi||^2) with E2 = -sum_{k < l anticommuting} h_l h_k P_l P_k the
 * second-order exponent: when K vanishes the error starts at
 * -(t^4 / (2 r^2)) ||E2 psi||^2.  Cached per handle for the last state.
 * Host only, O(L^2 ndet) (host threads for E2). */
int ps_ham_error_coefficient(ps_ham *ham, const uint64_t *idx, const double *amp, size_t ndet, double *out);

/* PS_MLP_FEATURES floats describing "first-order Trotter with r steps to
 * time t from psi" (t > 0, r >= 1; psi as for ps_ham_error_coefficient):
 *   log L, log lambda, log(max|h| / lambda), log t, log r, log C,
 *   log(C t^2 / r), one-norm fraction of diagonal terms (x = 0),
 *   log max(|K| / lambda^2, 1e-6),  log max(||E2 psi||^2 / lambda^4, 1e-6),
 *   log(e1 + e2) and e1 / (e1 + e2) for the error estimates e1 = |K| t^2 / r
 *   and e2 = ||E2 psi||^2 t^4 / (2 r^2) (the sum floored at 1e-6 lambda^2 t^2 / r),
 * C = ps_ham_trotter_bound(ham, L) (computed once per handle and cached).
 * PS_ERR_ARG when every pair of terms commutes (C = 0). Host only. */
int ps_ham_features(ps_ham *ham, const uint64_t *idx, const double *amp, size_t ndet, double t, uint32_t r,
                    float *out);

/* The first-order Trotter stream of ps_evolve_trotter: the term list r
 * times, angle (t / r) h_l; r * L rotations into the caller's arrays. */
int ps_trotter_stream(const ps_ham *ham, double t, uint32_t r, uint64_t *x_out, uint64_t *z_out, double *phi_out);

/* The plain doubling sweep: g_r = <psi0|U_r(t)|psi0> for r = 1, 2, 4, ...
 * (each evolved on `work` from a copy of psi0) until 2 |g_r - g_2r| <= eps;
 * *r_out = that r (0 if 2r would exceed r_max; then PS_ERR_UNSUPPORTED),
 * *rotations_out = rotations applied in total, g_out = g_r.  Synchronous. */
int ps_trotter_sweep(ps_state *work, const ps_state *psi0, const ps_ham *ham, double t, double eps, uint32_t r_max,
                     uint32_t *r_out, uint64_t *rotations_out, double *g_out);

typedef struct ps_mlp ps_mlp; /* opaque: network parameters and Adam state on one device */

/* Training knobs; zero selects the default. */
typedef struct ps_mlp_train_config {
    int epochs;      /* default 200 */
    int batch;       /* rows per Adam step (default 256); an epoch drops its last partial batch */
    float lr;        /* default 1e-3 */
    float beta1;     /* default 0.9 */
    float beta2;     /* default 0.999 */
    float eps;       /* default 1e-8 */
    uint64_t seed;   /* shuffling seed (SplitMix64 Fisher-Yates per epoch) */
} ps_mlp_train_config;

/* A network of n_in (1..16) inputs, three tanh hidden layers of 128 units
 * and one linear output, FP32, on the current device, ops on `stream`.
 * Parameters, flat and out-major (W[o][i] at o * fan_in + i):
 *   W1 (128 x n_in), b1 (128), W2 (128 x 128), b2, W3 (128 x 128), b3,
 *   w_out (128), b_out (1)   -- ps_mlp_num_params values.
 * Weights start Glorot-uniform from SplitMix64(seed), biases at zero.
 * Inputs are standardised per feature, (x - mu) / sigma, and the output is
 * y_mu + y_sigma * net(x); the loss of training is the mean squared error
 * of net(x) against (y - y_mu) / y_sigma. */
int ps_mlp_create(int n_in, uint64_t seed, void *stream, ps_mlp **out);
void ps_mlp_destroy(ps_mlp *m);
size_t ps_mlp_num_params(const ps_mlp *m);
int ps_mlp_get_params(ps_mlp *m, float *host);        /* synchronous */
int ps_mlp_set_params(ps_mlp *m, const float *host);  /* synchronous */
int ps_mlp_get_grads(ps_mlp *m, float *host);         /* gradient of the last ps_mlp_loss_grad */
int ps_mlp_set_grads(ps_mlp *m, const float *host);   /* replace it (an externally accumulated gradient for ps_mlp_adam_step) */
int ps_mlp_set_normalization(ps_mlp *m, const float *mu, const float *sigma, float y_mu, float y_sigma);
int ps_mlp_get_normalization(const ps_mlp *m, float *mu, float *sigma, float *y_mu, float *y_sigma);
/* mu and sigma (population standard deviation; 1 for a constant column) of
 * the host arrays x (rows x n_in, row-major) and y (rows). */
int ps_mlp_fit_normalization(ps_mlp *m, const float *x_host, const float *y_host, size_t rows);
/* Full-batch loss and gradient (kept on the device, read with
 * ps_mlp_get_grads) for device arrays x (rows x n_in) and y (rows). */
int ps_mlp_loss_grad(ps_mlp *m, const float *x_dev, const float *y_dev, size_t rows, double *loss_out);
/* One Adam step (Kingma & Ba, bias-corrected) with the current gradient. */
int ps_mlp_adam_step(ps_mlp *m, float lr, float beta1, float beta2, float eps);
/* Mini-batch Adam on device arrays; every epoch is one CUDA graph replay.
 * loss_per_epoch (epochs floats, may be NULL) receives the mean training
 * loss of each epoch (synchronising once per epoch). */
int ps_mlp_train(ps_mlp *m, const float *x_dev, const float *y_dev, size_t rows, const ps_mlp_train_config *cfg,
                 float *loss_per_epoch);
/* y_dev[i] = the network's prediction for row i of x_dev (asynchronous). */
int ps_mlp_predict(ps_mlp *m, const float *x_dev, size_t rows, float *y_dev);
/* Smallest r in 1..r_max whose predicted log error (a network trained on
 * log eps with ps_ham_features inputs for the initial state psi) is
 * <= log(eps) - margin; pred_out (r_max floats, may be NULL) receives every
 * prediction.  PS_ERR_UNSUPPORTED (r_out = 0) when no r qualifies.
 * Synchronous. */
int ps_mlp_pick_r(ps_mlp *m, ps_ham *ham, const uint64_t *idx, const double *amp, size_t ndet, double t, double eps,
                  double margin, uint32_t r_max, uint32_t *r_out, float *pred_out);
/* The ensemble's prediction for `rows` device feature rows: the mean, in
 * member order (FP64 sum, rounded once to FP32), of every member's
 * predicted log error, written to host memory y_host.  Synchronous. */
int ps_mlp_predict_ensemble(ps_mlp *const *nets, int count, const float *x_dev, size_t rows, float *y_host);

/* The same for an ensemble of `count` (1..64) networks on one device: the
 * prediction is the mean of the members' predicted log errors. */
int ps_mlp_pick_r_ensemble(ps_mlp *const *nets, int count, ps_ham *ham, const uint64_t *idx, const double *amp,
                           size_t ndet, double t, double eps, double margin, uint32_t r_max, uint32_t *r_out,
                           float *pred_out);

#ifdef __cplusplus
}
#endif

#endif /* PS_H */
