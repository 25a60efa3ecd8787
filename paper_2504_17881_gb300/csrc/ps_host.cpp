// libps C ABI: state handles, plan upload and launch, reductions,
// Hamiltonians and product-formula drivers.  See include/ps.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "ps_internal.h"
#include "ps_sample.h"

namespace ps {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

static int fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

static int cuda_fail(cudaError_t e, const char *what) {
    std::ostringstream os;
    os << what << ": " << cudaGetErrorName(e) << " (" << cudaGetErrorString(e) << ")";
    return fail(PS_ERR_CUDA, os.str());
}

#define PS_CUDA(call, what)                      \
    do {                                         \
        cudaError_t e__ = (call);                \
        if (e__ != cudaSuccess) return cuda_fail(e__, what); \
    } while (0)

// Kernel parameters of one window, read from the host copy of the plan.
void fill_tile_params(const Plan &p, const WinDesc &w, TileParams &tp) {
    std::memset(&tp, 0, sizeof(tp));
    for (int i = 0; i < w.d; ++i) {
        tp.v[i] = w.v[i];
        tp.piv[i] = w.piv[i];
    }
    tp.c = w.c;
    tp.d = w.d;
    tp.nsub = w.nsub;
    tp.nrot = w.nrot;
    for (int s = 0; s < w.nsub; ++s) {
        const SubDesc &sd = p.sub[w.sub_off + s];
        for (int i = 0; i < kMaxG; ++i) {
            tp.sub[s].u[i] = sd.u[i];
            tp.sub[s].piv[i] = sd.piv[i];
        }
        tp.sub[s].r0 = (uint8_t)(sd.rot_off - w.rot_off);
        tp.sub[s].r1 = (uint8_t)(sd.rot_off - w.rot_off + sd.nrot);
        tp.sub[s].fast = sd.fast;
        tp.sub[s].pad = 0;
    }
    for (int r = 0; r < w.nrot; ++r) {
        const RotDesc &rd = p.rot[w.rot_off + r];
        TileRotP &rp = tp.rot[r];
        rp.base = rd.base64;
        rp.c = rd.c64;
        rp.z = rd.z;
        rp.zt = rd.zt;
        rp.smask = rd.smask;
        rp.meta = (uint32_t)rd.mu | ((uint32_t)(rd.flags & 1) << 5) | ((uint32_t)((rd.flags >> 1) & 1) << 6);
    }
}

static void fill_pair_params(const Plan &p, const WinDesc &w, PairParams &pp) {
    const RotDesc &rd = p.rot[w.rot_off];
    pp.x = rd.x;
    pp.z = rd.z;
    pp.base = rd.base64;
    pp.c = rd.c64;
    pp.flags = rd.flags;
    pp.pad = 0;
}

struct TimedLaunch {
    int kind;
    cudaEvent_t a, b;
};

}  // namespace ps

using namespace ps;

struct ps_state {
    int n = 0;
    int dtype = 0;
    void *psi = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    Tuning tun{};
    // reductions
    double *partials = nullptr;
    double *rout = nullptr;
    double *hout = nullptr;
    // The stored amplitudes equal the evolved state divided by `pending`:
    // cos(phi) factors of tangent-form rotations are applied per pass only to
    // the precision the storage type holds, the rest is carried here (FP64)
    // and folded into later passes and into ps_norm / ps_overlap.
    double pending = 1.0;
    // statistics
    ps_stats stats{};
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> event_pool;
};


struct ps_plan {
    Plan plan;  // host copy; every launch passes its window by value
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t state_bytes(const ps_state *st) { return ((size_t)(st->dtype == PS_C64 ? 8 : 16)) << st->n; }

cudaEvent_t get_event(ps_state *st) {
    if (!st->event_pool.empty()) {
        cudaEvent_t e = st->event_pool.back();
        st->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Drain recorded launch timings into the counters.
int collect_timings(ps_state *st) {
    if (st->timed.empty()) return PS_OK;
    PS_CUDA(cudaStreamSynchronize(st->stream), "cudaStreamSynchronize");
    for (auto &t : st->timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) st->stats.kernel_ms[t.kind] += ms;
        st->event_pool.push_back(t.a);
        st->event_pool.push_back(t.b);
    }
    st->timed.clear();
    return PS_OK;
}

// Raise the dynamic shared-memory limit of every tile-kernel instance once
// per device (the limit is an upper bound; each launch asks for what it uses).
int ensure_prepared(ps_state *st) {
    static std::mutex mu;
    static std::vector<int> done(2 * 64, 0);
    std::lock_guard<std::mutex> lock(mu);
    const int slot = 2 * (st->device & 63) + st->dtype;
    if (done[slot]) return PS_OK;
    int e = prepare_kernels(st->dtype);
    if (e != 0) return cuda_fail((cudaError_t)e, "cudaFuncSetAttribute (tile kernel shared memory)");
    done[slot] = 1;
    return PS_OK;
}

// Launch every window of a plan on the state's stream.
int launch_plan(ps_state *st, const Plan &p) {
    if (p.win.empty()) return PS_OK;
    int rc = ensure_prepared(st);
    if (rc) return rc;
    const bool timing = st->tun.kernel_timing != 0;
    const double pass_bytes = 2.0 * (double)state_bytes(st);
    TileParams tp;
    PairParams pp;
    for (size_t wi = 0; wi < p.win.size(); ++wi) {
        const WinDesc &w = p.win[wi];
        const int kind = w.kind == 1 ? PS_KERNEL_PAIR : PS_KERNEL_TILE;
        cudaEvent_t ea = nullptr, eb = nullptr;
        if (timing) {
            ea = get_event(st);
            eb = get_event(st);
            if (!ea || !eb) return fail(PS_ERR_CUDA, "cudaEventCreate failed");
            PS_CUDA(cudaEventRecord(ea, st->stream), "cudaEventRecord");
        }
        // Carry the window's cos(phi) product; apply it as a <- a + kdelta a
        // (one rounding, unbiased) once it is far enough from 1: beyond 2^-16
        // for complex64, where a factor within an ulp of 1 would round away
        // systematically, and beyond 2^-20 for complex128, whose FP64 pass is
        // bound by its FP64 arithmetic (applying the factor every pass would
        // add two FMAs per amplitude to about eighteen).  Until then the
        // stored amplitudes are the state divided by the carried factor.
        st->pending *= w.kprod;
        double kdelta = 0.0;
        const double dev = st->pending - 1.0;
        if (st->dtype == PS_C128) {
            if (std::fabs(dev) > 0x1.0p-20) kdelta = dev;
        } else if (std::fabs(dev) > 0x1.0p-16) {
            kdelta = (double)(float)dev;
        }
        if (kdelta != 0.0) st->pending /= (1.0 + kdelta);
        int e;
        if (w.kind == 1) {
            fill_pair_params(p, w, pp);
            e = launch_pair(st->dtype, st->psi, st->n, pp, kdelta, st->stream, st->num_sms);
        } else {
            fill_tile_params(p, w, tp);
            e = launch_tile(st->dtype, p.G, p.NG, st->psi, st->n, tp, kdelta, st->stream, p.threads);
        }
        if (e != 0) return cuda_fail((cudaError_t)e, w.kind == 1 ? "pair kernel launch" : "tile kernel launch");
        if (timing) {
            PS_CUDA(cudaEventRecord(eb, st->stream), "cudaEventRecord");
            st->timed.push_back({kind, ea, eb});
        }
        st->stats.launches[kind] += 1;
        st->stats.bytes[kind] += pass_bytes;
        st->stats.passes += 1;
        st->stats.rotations += (uint64_t)w.nrot;
    }
    if (timing && st->timed.size() > 65536) return collect_timings(st);
    return PS_OK;
}

// Schedule on the host and launch.
int run_sequence(ps_state *st, const uint64_t *x, const uint64_t *z, const double *phi, size_t count) {
    if (count == 0) return PS_OK;
    Plan p;
    std::string err;
    int rc = build_plan(st->n, st->dtype, x, z, phi, count, st->tun, p, &err);
    if (rc) return fail(rc, err);
    return launch_plan(st, p);
}

int check_state(const ps_state *st) {
    if (!st) return fail(PS_ERR_ARG, "null state handle");
    return PS_OK;
}

int reduce(ps_state *st, int what, const void *a, const void *b, double out[2]) {
    const bool timing = st->tun.kernel_timing != 0;
    cudaEvent_t ea = nullptr, eb = nullptr;
    if (timing) {
        ea = get_event(st);
        eb = get_event(st);
        if (!ea || !eb) return fail(PS_ERR_CUDA, "cudaEventCreate failed");
        PS_CUDA(cudaEventRecord(ea, st->stream), "cudaEventRecord");
    }
    int e = launch_reduce(st->dtype, what, a, b, st->n, st->partials, st->rout, st->stream);
    if (e) return cuda_fail((cudaError_t)e, "reduction launch");
    if (timing) {
        PS_CUDA(cudaEventRecord(eb, st->stream), "cudaEventRecord");
        st->timed.push_back({PS_KERNEL_REDUCE, ea, eb});
    }
    st->stats.launches[PS_KERNEL_REDUCE] += 2;
    st->stats.bytes[PS_KERNEL_REDUCE] += (double)state_bytes(st) * (what == 0 ? 1.0 : 2.0);
    PS_CUDA(cudaMemcpyAsync(st->hout, st->rout, 2 * sizeof(double), cudaMemcpyDeviceToHost, st->stream),
            "reduction readback");
    PS_CUDA(cudaStreamSynchronize(st->stream), "cudaStreamSynchronize");
    out[0] = st->hout[0];
    out[1] = st->hout[1];
    return PS_OK;
}

int validate_masks(int n, size_t L, const uint64_t *x, const uint64_t *z) {
    for (size_t l = 0; l < L; ++l)
        if ((x[l] | z[l]) >> n) {
            std::ostringstream os;
            os << "term " << l << " has a mask bit >= n=" << n;
            return fail(PS_ERR_ARG, os.str());
        }
    return PS_OK;
}

}  // namespace

extern "C" {

const char *ps_last_error(void) { return g_err.c_str(); }

int ps_abi_version(void) { return 3; }

int ps_device_count(void) {
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) return -1;
    return n;
}

int ps_create(int n, int dtype, void *dev_state, void *stream, ps_state **out) {
    if (!out) return fail(PS_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (n < 1 || n > kMaxN) return fail(PS_ERR_ARG, "n must be in [1, 40]");
    if (dtype != PS_C64 && dtype != PS_C128) return fail(PS_ERR_ARG, "dtype must be PS_C64 or PS_C128");
    if (!dev_state) return fail(PS_ERR_ARG, "null state buffer (the caller owns the 2^n amplitudes)");
    if (((uintptr_t)dev_state) & 15) return fail(PS_ERR_ARG, "state buffer must be 16-byte aligned");
    ps_state *st = new (std::nothrow) ps_state();
    if (!st) return fail(PS_ERR_OOM, "host allocation failed");
    st->n = n;
    st->dtype = dtype;
    st->psi = dev_state;
    st->stream = (cudaStream_t)stream;
    st->tun = resolve_tuning(nullptr, dtype);
    cudaError_t e = cudaGetDevice(&st->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&st->num_sms, cudaDevAttrMultiProcessorCount, st->device);
    if (e == cudaSuccess) e = cudaMalloc((void **)&st->partials, 2 * sizeof(double) * (size_t)reduce_blocks());
    if (e == cudaSuccess) e = cudaMalloc((void **)&st->rout, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&st->hout, 2 * sizeof(double));
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "ps_create");
        ps_destroy(st);
        return rc;
    }
    *out = st;
    return PS_OK;
}

void ps_destroy(ps_state *st) {
    if (!st) return;
    DeviceGuard g(st->device);
    cudaStreamSynchronize(st->stream);
    for (auto &t : st->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : st->event_pool) cudaEventDestroy(e);
    if (st->partials) cudaFree(st->partials);
    if (st->rout) cudaFree(st->rout);
    if (st->hout) cudaFreeHost(st->hout);
    delete st;
}

int ps_set_state(ps_state *st, const void *host_src) {
    if (int rc = check_state(st)) return rc;
    if (!host_src) return fail(PS_ERR_ARG, "null host buffer");
    DeviceGuard g(st->device);
    PS_CUDA(cudaMemcpyAsync(st->psi, host_src, state_bytes(st), cudaMemcpyHostToDevice, st->stream), "ps_set_state");
    st->pending = 1.0;
    return PS_OK;
}

int ps_get_state(ps_state *st, void *host_dst) {
    if (int rc = check_state(st)) return rc;
    if (!host_dst) return fail(PS_ERR_ARG, "null host buffer");
    DeviceGuard g(st->device);
    PS_CUDA(cudaMemcpyAsync(host_dst, st->psi, state_bytes(st), cudaMemcpyDeviceToHost, st->stream), "ps_get_state");
    PS_CUDA(cudaStreamSynchronize(st->stream), "cudaStreamSynchronize");
    return PS_OK;
}

int ps_get_state_represented(ps_state *st, void *host_dst) {
    if (int rc = check_state(st)) return rc;
    if (!host_dst) return fail(PS_ERR_ARG, "null host buffer");
    DeviceGuard g(st->device);
    // the stored amplitudes land in the front of the buffer; complex64 ones are
    // widened in place from the last element down (element i's 16 output bytes
    // start at or above byte 16 i, so no unread input is overwritten)
    PS_CUDA(cudaMemcpyAsync(host_dst, st->psi, state_bytes(st), cudaMemcpyDeviceToHost, st->stream),
            "ps_get_state_represented");
    PS_CUDA(cudaStreamSynchronize(st->stream), "cudaStreamSynchronize");
    const uint64_t N = 1ull << st->n;
    const double f = st->pending;
    double *out = static_cast<double *>(host_dst);
    if (st->dtype == PS_C64) {
        const float *in = static_cast<const float *>(host_dst);
        for (uint64_t i = N; i-- > 0;) {
            const double re = (double)in[2 * i], im = (double)in[2 * i + 1];
            out[2 * i] = f * re;
            out[2 * i + 1] = f * im;
        }
    } else if (f != 1.0) {
        for (uint64_t i = 0; i < 2 * N; ++i) out[i] *= f;
    }
    return PS_OK;
}

int ps_copy_state(ps_state *dst, const ps_state *src) {
    if (int rc = check_state(dst)) return rc;
    if (int rc = check_state(src)) return rc;
    if (dst->n != src->n || dst->dtype != src->dtype) return fail(PS_ERR_ARG, "states differ in n or dtype");
    DeviceGuard g(dst->device);
    PS_CUDA(cudaMemcpyAsync(dst->psi, src->psi, state_bytes(dst), cudaMemcpyDeviceToDevice, dst->stream),
            "ps_copy_state");
    dst->pending = src->pending;
    return PS_OK;
}

int ps_set_tuning(ps_state *st, const ps_tuning *tuning) {
    if (int rc = check_state(st)) return rc;
    Tuning t = resolve_tuning(tuning, st->dtype);
    Plan probe;
    std::string err;
    uint64_t zero = 0;
    double ang = 0.0;
    int rc = build_plan(st->n, st->dtype, &zero, &zero, &ang, 1, t, probe, &err);
    if (rc) return fail(rc, err);
    st->tun = t;
    return PS_OK;
}

int ps_apply_rotations(ps_state *st, const uint64_t *x, const uint64_t *z, const double *phi, size_t count) {
    if (int rc = check_state(st)) return rc;
    if (count == 0) return PS_OK;
    DeviceGuard g(st->device);
    return run_sequence(st, x, z, phi, count);
}

int ps_plan_create(int n, int dtype, const uint64_t *x, const uint64_t *z, const double *phi, size_t count,
                   const ps_tuning *tuning, ps_plan **out) {
    if (!out) return fail(PS_ERR_ARG, "null output pointer");
    *out = nullptr;
    ps_plan *pl = new (std::nothrow) ps_plan();
    if (!pl) return fail(PS_ERR_OOM, "host allocation failed");
    std::string err;
    int rc = build_plan(n, dtype, x, z, phi, count, resolve_tuning(tuning, dtype), pl->plan, &err);
    if (rc) {
        delete pl;
        return fail(rc, err);
    }
    *out = pl;
    return PS_OK;
}

int ps_plan_apply(ps_state *st, const ps_plan *plan) {
    if (int rc = check_state(st)) return rc;
    if (!plan) return fail(PS_ERR_ARG, "null plan");
    if (plan->plan.n != st->n || plan->plan.dtype != st->dtype) return fail(PS_ERR_ARG, "plan built for another n or dtype");
    DeviceGuard g(st->device);
    return launch_plan(st, plan->plan);
}

static void fill_info(const Plan &p, ps_plan_info *out) {
    std::memset(out, 0, sizeof(*out));
    out->rotations = p.rotations;
    out->windows = p.win.size();
    for (const auto &w : p.win) {
        if (w.kind == 1)
            out->pair_windows++;
        else {
            out->tile_windows++;
            out->subwindows += (uint64_t)w.nsub;
            for (int si = 0; si < w.nsub; ++si) out->fast_subwindows += p.sub[w.sub_off + si].fast ? 1 : 0;
        }
        out->max_window = std::max<uint64_t>(out->max_window, (uint64_t)w.nrot);
    }
    out->tile_bits = p.B;
    out->group_bits = p.G;
}

int ps_plan_get_info(const ps_plan *plan, ps_plan_info *out) {
    if (!plan || !out) return fail(PS_ERR_ARG, "null argument");
    fill_info(plan->plan, out);
    return PS_OK;
}

void ps_plan_destroy(ps_plan *plan) { delete plan; }

int ps_plan_describe(int n, int dtype, const uint64_t *x, const uint64_t *z, const double *phi, size_t count,
                     const ps_tuning *tuning, ps_plan_info *out) {
    if (!out) return fail(PS_ERR_ARG, "null output pointer");
    Plan p;
    std::string err;
    int rc = build_plan(n, dtype, x, z, phi, count, resolve_tuning(tuning, dtype), p, &err);
    if (rc) return fail(rc, err);
    fill_info(p, out);
    return PS_OK;
}

int ps_plan_export(int n, int dtype, const uint64_t *x, const uint64_t *z, const double *phi, size_t count,
                   const ps_tuning *tuning, size_t max_windows, size_t *n_windows, uint32_t *window_of, uint32_t *xt,
                   uint32_t *zt, int *kind, int *c, int *d, uint64_t *basis) {
    if (!n_windows) return fail(PS_ERR_ARG, "null output pointer");
    Plan p;
    std::string err;
    int rc = build_plan(n, dtype, x, z, phi, count, resolve_tuning(tuning, dtype), p, &err);
    if (rc) return fail(rc, err);
    *n_windows = p.win.size();
    if (p.win.size() > max_windows) return fail(PS_ERR_ARG, "max_windows too small");
    if (count && (!window_of || !xt || !zt)) return fail(PS_ERR_ARG, "null per-rotation output");
    if (!p.win.empty() && (!kind || !c || !d || !basis)) return fail(PS_ERR_ARG, "null per-window output");
    for (size_t wi = 0; wi < p.win.size(); ++wi) {
        const WinDesc &w = p.win[wi];
        kind[wi] = w.kind;
        c[wi] = w.c;
        d[wi] = w.d;
        for (int i = 0; i < 16; ++i) basis[wi * 16 + i] = i < w.d ? w.v[i] : 0;
        for (int r = 0; r < w.nrot; ++r) window_of[w.rot_off + r] = (uint32_t)wi;
    }
    // tile-local masks: recover x~ from the register-stage coordinates
    for (const WinDesc &w : p.win) {
        for (int r = 0; r < w.nrot; ++r) {
            xt[w.rot_off + r] = 0;
            zt[w.rot_off + r] = 0;
        }
        if (w.kind == 1) continue;
        for (int si = 0; si < w.nsub; ++si) {
            const SubDesc &sd = p.sub[w.sub_off + si];
            for (int r = sd.rot_off; r < sd.rot_off + sd.nrot; ++r) {
                const RotDesc &rd = p.rot[r];
                uint32_t v = 0;
                for (int i = 0; i < p.G; ++i)
                    if ((rd.mu >> i) & 1) v ^= sd.u[i];
                xt[r] = v;
                zt[r] = rd.zt;
            }
        }
    }
    return PS_OK;
}

int ps_norm(ps_state *st, double *out) {
    if (int rc = check_state(st)) return rc;
    if (!out) return fail(PS_ERR_ARG, "null output pointer");
    DeviceGuard g(st->device);
    double r[2];
    int rc = reduce(st, 0, st->psi, nullptr, r);
    if (rc) return rc;
    *out = r[0] * st->pending * st->pending;
    return PS_OK;
}

int ps_overlap(const ps_state *psi0, ps_state *psi, double out[2]) {
    if (int rc = check_state(psi0)) return rc;
    if (int rc = check_state(psi)) return rc;
    if (!out) return fail(PS_ERR_ARG, "null output pointer");
    if (psi0->n != psi->n || psi0->dtype != psi->dtype) return fail(PS_ERR_ARG, "states differ in n or dtype");
    DeviceGuard g(psi->device);
    if (psi0->stream != psi->stream) {
        cudaEvent_t e = nullptr;
        PS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
        cudaEventRecord(e, psi0->stream);
        cudaStreamWaitEvent(psi->stream, e, 0);
        cudaEventDestroy(e);
    }
    int rc = reduce(psi, 1, psi0->psi, psi->psi, out);
    if (rc) return rc;
    const double f = psi0->pending * psi->pending;
    out[0] *= f;
    out[1] *= f;
    return PS_OK;
}

int ps_get_scale(const ps_state *st, double *out) {
    if (int rc = check_state(st)) return rc;
    if (!out) return fail(PS_ERR_ARG, "null output pointer");
    *out = st->pending;
    return PS_OK;
}

int ps_ham_create(int n, size_t L, const uint64_t *x, const uint64_t *z, const double *h, ps_ham **out) {
    if (!out) return fail(PS_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (n < 1 || n > kMaxN) return fail(PS_ERR_ARG, "n must be in [1, 40]");
    if (L == 0) return fail(PS_ERR_ARG, "a Hamiltonian needs at least one term");
    if (!x || !z || !h) return fail(PS_ERR_ARG, "null term array");
    if (int rc = validate_masks(n, L, x, z)) return rc;
    for (size_t l = 0; l < L; ++l)
        if (!std::isfinite(h[l])) return fail(PS_ERR_ARG, "non-finite coefficient");
    ps_ham *H = new (std::nothrow) ps_ham();
    if (!H) return fail(PS_ERR_OOM, "host allocation failed");
    H->H.n = n;
    H->H.x.assign(x, x + L);
    H->H.z.assign(z, z + L);
    H->H.h.assign(h, h + L);
    *out = H;
    return PS_OK;
}

void ps_ham_destroy(ps_ham *ham) { delete ham; }

double ps_ham_lambda(const ps_ham *ham) { return ham ? ham_lambda(ham->H) : 0.0; }

int ps_qdrift_stream(const ps_ham *ham, double t, uint64_t N, uint64_t seed, uint64_t first, uint64_t count,
                     uint64_t *x_out, uint64_t *z_out, double *phi_out) {
    if (!ham) return fail(PS_ERR_ARG, "null Hamiltonian");
    if (N == 0) return fail(PS_ERR_ARG, "qDRIFT needs N >= 1");
    if (count && (!x_out || !z_out || !phi_out)) return fail(PS_ERR_ARG, "null output array");
    std::string err;
    int rc = qdrift_stream(ham->H, t, N, seed, first, count, x_out, z_out, phi_out, &err);
    if (rc) return fail(rc, err);
    return PS_OK;
}

uint64_t ps_partial_length(const ps_ham *ham, size_t L_D, uint32_t r, uint64_t Ns) {
    if (!ham || L_D > ham->H.h.size()) return 0;
    return partial_length(ham->H, L_D, r, Ns);
}

int ps_partial_stream(const ps_ham *ham, size_t L_D, double t, uint32_t r, uint64_t Ns, uint64_t seed,
                      uint64_t *x_out, uint64_t *z_out, double *phi_out) {
    if (!ham) return fail(PS_ERR_ARG, "null Hamiltonian");
    if (r == 0) return fail(PS_ERR_ARG, "r must be >= 1");
    if (L_D > ham->H.h.size()) return fail(PS_ERR_ARG, "L_D exceeds the number of terms");
    Stream s;
    partial_stream(ham->H, L_D, t, r, Ns, seed, s);
    if (s.size() && (!x_out || !z_out || !phi_out)) return fail(PS_ERR_ARG, "null output array");
    std::copy(s.x.begin(), s.x.end(), x_out);
    std::copy(s.z.begin(), s.z.end(), z_out);
    std::copy(s.phi.begin(), s.phi.end(), phi_out);
    return PS_OK;
}

int ps_evolve_trotter(ps_state *st, const ps_ham *ham, double t, uint32_t r) {
    if (int rc = check_state(st)) return rc;
    if (!ham) return fail(PS_ERR_ARG, "null Hamiltonian");
    if (ham->H.n != st->n) return fail(PS_ERR_ARG, "Hamiltonian and state differ in n");
    if (r == 0) return fail(PS_ERR_ARG, "r must be >= 1");
    Stream s;
    trotter_stream(ham->H, t, r, s);
    DeviceGuard g(st->device);
    return run_sequence(st, s.x.data(), s.z.data(), s.phi.data(), s.size());
}

int ps_evolve_qdrift(ps_state *st, const ps_ham *ham, double t, uint64_t N, uint64_t seed) {
    if (int rc = check_state(st)) return rc;
    if (!ham) return fail(PS_ERR_ARG, "null Hamiltonian");
    if (ham->H.n != st->n) return fail(PS_ERR_ARG, "Hamiltonian and state differ in n");
    if (N == 0) return fail(PS_ERR_ARG, "qDRIFT needs N >= 1");
    Stream s;
    s.resize((size_t)N);
    std::string err;
    int rc = qdrift_stream(ham->H, t, N, seed, 0, N, s.x.data(), s.z.data(), s.phi.data(), &err);
    if (rc) return fail(rc, err);
    DeviceGuard g(st->device);
    return run_sequence(st, s.x.data(), s.z.data(), s.phi.data(), s.size());
}

int ps_evolve_partial(ps_state *st, const ps_ham *ham, size_t L_D, double t, uint32_t r, uint64_t Ns,
                      uint64_t seed) {
    if (int rc = check_state(st)) return rc;
    if (!ham) return fail(PS_ERR_ARG, "null Hamiltonian");
    if (ham->H.n != st->n) return fail(PS_ERR_ARG, "Hamiltonian and state differ in n");
    if (r == 0) return fail(PS_ERR_ARG, "r must be >= 1");
    if (L_D > ham->H.h.size()) return fail(PS_ERR_ARG, "L_D exceeds the number of terms");
    Stream s;
    partial_stream(ham->H, L_D, t, r, Ns, seed, s);
    DeviceGuard g(st->device);
    return run_sequence(st, s.x.data(), s.z.data(), s.phi.data(), s.size());
}

int ps_evolve_trotter2(ps_state *st, const ps_ham *ham, double t, uint32_t r) {
    if (int rc = check_state(st)) return rc;
    if (!ham) return fail(PS_ERR_ARG, "null Hamiltonian");
    if (ham->H.n != st->n) return fail(PS_ERR_ARG, "Hamiltonian and state differ in n");
    if (r == 0) return fail(PS_ERR_ARG, "r must be >= 1");
    Stream s;
    trotter2_stream(ham->H, t, r, s);
    DeviceGuard g(st->device);
    return run_sequence(st, s.x.data(), s.z.data(), s.phi.data(), s.size());
}

int ps_evolve_partial2(ps_state *st, const ps_ham *ham, size_t L_D, double t, uint32_t r, uint64_t Ns,
                       uint64_t seed) {
    if (int rc = check_state(st)) return rc;
    if (!ham) return fail(PS_ERR_ARG, "null Hamiltonian");
    if (ham->H.n != st->n) return fail(PS_ERR_ARG, "Hamiltonian and state differ in n");
    if (r == 0) return fail(PS_ERR_ARG, "r must be >= 1");
    if (L_D > ham->H.h.size()) return fail(PS_ERR_ARG, "L_D exceeds the number of terms");
    Stream s;
    partial2_stream(ham->H, L_D, t, r, Ns, seed, s);
    DeviceGuard g(st->device);
    return run_sequence(st, s.x.data(), s.z.data(), s.phi.data(), s.size());
}

uint64_t ps_trotter2_length(const ps_ham *ham, uint32_t r) { return ham ? trotter2_length(ham->H.h.size(), r) : 0; }

int ps_trotter2_stream(const ps_ham *ham, double t, uint32_t r, uint64_t *x_out, uint64_t *z_out, double *phi_out) {
    if (!ham) return fail(PS_ERR_ARG, "null Hamiltonian");
    if (r == 0) return fail(PS_ERR_ARG, "r must be >= 1");
    Stream s;
    trotter2_stream(ham->H, t, r, s);
    if (s.size() && (!x_out || !z_out || !phi_out)) return fail(PS_ERR_ARG, "null output array");
    std::copy(s.x.begin(), s.x.end(), x_out);
    std::copy(s.z.begin(), s.z.end(), z_out);
    std::copy(s.phi.begin(), s.phi.end(), phi_out);
    return PS_OK;
}

uint64_t ps_partial2_length(const ps_ham *ham, size_t L_D, uint32_t r, uint64_t Ns) {
    if (!ham || L_D > ham->H.h.size()) return 0;
    return partial2_length(ham->H, L_D, r, Ns);
}

int ps_partial2_stream(const ps_ham *ham, size_t L_D, double t, uint32_t r, uint64_t Ns, uint64_t seed,
                       uint64_t *x_out, uint64_t *z_out, double *phi_out) {
    if (!ham) return fail(PS_ERR_ARG, "null Hamiltonian");
    if (r == 0) return fail(PS_ERR_ARG, "r must be >= 1");
    if (L_D > ham->H.h.size()) return fail(PS_ERR_ARG, "L_D exceeds the number of terms");
    Stream s;
    partial2_stream(ham->H, L_D, t, r, Ns, seed, s);
    if (s.size() && (!x_out || !z_out || !phi_out)) return fail(PS_ERR_ARG, "null output array");
    std::copy(s.x.begin(), s.x.end(), x_out);
    std::copy(s.z.begin(), s.z.end(), z_out);
    std::copy(s.phi.begin(), s.phi.end(), phi_out);
    return PS_OK;
}

int ps_ham_sort_lexicographic(ps_ham *ham) {
    if (!ham) return fail(PS_ERR_ARG, "null Hamiltonian");
    lexicographic_sort(ham->H);
    ham->k_valid = false;  // the error coefficients depend on the term order
    return PS_OK;
}

int ps_get_stats(ps_state *st, ps_stats *out) {
    if (int rc = check_state(st)) return rc;
    if (!out) return fail(PS_ERR_ARG, "null output pointer");
    DeviceGuard g(st->device);
    if (int rc = collect_timings(st)) return rc;
    *out = st->stats;
    return PS_OK;
}

int ps_reset_stats(ps_state *st) {
    if (int rc = check_state(st)) return rc;
    DeviceGuard g(st->device);
    if (int rc = collect_timings(st)) return rc;
    std::memset(&st->stats, 0, sizeof(st->stats));
    return PS_OK;
}

}  // extern "C"
