// Host side of the batched persistent launch (see include/ps.h and
// ps_batch.cu): per-run schedules built in parallel threads, windows packed
// for the device, lanes filled longest-first, and one cooperative launch
// captured in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <queue>
#include <sstream>
#include <string>
#include <thread>
#include <unordered_set>
#include <vector>

#include "ps_internal.h"

namespace ps {
namespace {

int bfail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

int cuda_bfail(cudaError_t e, const char *what) {
    std::ostringstream os;
    os << what << ": " << cudaGetErrorName(e) << " (" << cudaGetErrorString(e) << ")";
    return bfail(e == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA, os.str());
}

struct BatchCfg {
    int lane_size, lane_log, tile_bits, resident_bits, single_bits, use_graph, wait_ms, withhold;
};

constexpr int kTileFloor = 8;

int resolve_cfg(int dtype, const ps_batch_config *c, BatchCfg &r) {
    const int bmax = dtype == PS_C64 ? 13 : 12;
    r.lane_size = (c && c->lane_size) ? c->lane_size : 16;
    if (r.lane_size < 1 || r.lane_size > 256 || (r.lane_size & (r.lane_size - 1)))
        return bfail(PS_ERR_ARG, "lane_size must be a power of two in [1, 256]");
    r.lane_log = 31 - __builtin_clz((unsigned)r.lane_size);
    r.tile_bits = (c && c->tile_bits) ? c->tile_bits : bmax;
    if (r.tile_bits < kTileFloor || r.tile_bits > bmax)
        return bfail(PS_ERR_ARG, dtype == PS_C64 ? "tile_bits must be in [8, 13] for PS_C64"
                                                 : "tile_bits must be in [8, 12] for PS_C128");
    r.resident_bits = (c && c->resident_bits) ? c->resident_bits : bmax;
    if (r.resident_bits != -1 && (r.resident_bits < 1 || r.resident_bits > bmax))
        return bfail(PS_ERR_ARG, "resident_bits must be -1 or in [1, 13] (PS_C64) / [1, 12] (PS_C128)");
    const int res = r.resident_bits < 0 ? 0 : r.resident_bits;
    r.single_bits = (c && c->single_bits) ? c->single_bits : res + 1;
    if (r.single_bits != -1 && (r.single_bits < 1 || r.single_bits > 30))
        return bfail(PS_ERR_ARG, "single_bits must be -1 or in [1, 30]");
    r.use_graph = (c && c->use_graph) ? c->use_graph : 1;
    if (r.use_graph != 1 && r.use_graph != -1) return bfail(PS_ERR_ARG, "use_graph must be 0, 1 or -1");
    r.wait_ms = (c && c->wait_ms) ? c->wait_ms : 5000;
    if (r.wait_ms < 1 || r.wait_ms > 600000) return bfail(PS_ERR_ARG, "wait_ms must be in [1, 600000]");
    r.withhold = c ? c->test_withhold : 0;
    if (r.withhold != 0 && r.withhold != 1) return bfail(PS_ERR_ARG, "test_withhold must be 0 or 1");
    return PS_OK;
}

// The schedule of a whole batch, independent of device pointers.
struct Layout {
    std::vector<BatchRun> runs;
    std::vector<BatchWin> wins;
    std::vector<unsigned char> bodies;
    std::vector<int> lane_runs, lane_off, single_order;
    std::vector<double> work;  // per run: 2^n x (windows + 1)
    size_t smem = 0;
    int nlanes = 0;
    ps_batch_info info{};
};

size_t amp_bytes(int dtype) { return dtype == PS_C64 ? 8 : 16; }

// Tile bits of run n for the configuration (kind: -2 resident, -1 single, 0 lane).
int run_tile_bits(int n, int kind, const BatchCfg &c) {
    if (kind == -2) return n;
    int B = kind == -1 ? c.tile_bits : std::max(kTileFloor, n - c.lane_log);
    B = std::min(B, c.tile_bits);
    return std::min(B, n);
}

// Pack window w of plan p: head, rounds (padded to 8 bytes), rotations.
void pack_window(const Plan &p, const WinDesc &w, std::vector<unsigned char> &out) {
    TileParams tp;
    fill_tile_params(p, w, tp);
    const size_t sub_bytes = ((size_t)w.nsub * sizeof(TileSubP) + 7) & ~(size_t)7;
    const size_t at = out.size();
    out.resize(at + kWinHeadBytes + sub_bytes + (size_t)w.nrot * sizeof(TileRotP), 0);
    unsigned char *d = out.data() + at;
    std::memcpy(d, &tp, kWinHeadBytes);
    std::memcpy(d + kWinHeadBytes, tp.sub, (size_t)w.nsub * sizeof(TileSubP));
    std::memcpy(d + kWinHeadBytes + sub_bytes, tp.rot, (size_t)w.nrot * sizeof(TileRotP));
}

// Validate the runs, schedule each on the host (in parallel), pack the
// windows and fill the lanes for a grid of `grid` CTAs.
int build_layout(int dtype, const ps_run_desc *runs, size_t nruns, const BatchCfg &cfg, int grid, bool need_ptrs,
                 Layout &L) {
    if (dtype != PS_C64 && dtype != PS_C128) return bfail(PS_ERR_ARG, "dtype must be PS_C64 or PS_C128");
    if (nruns == 0) return bfail(PS_ERR_ARG, "a batch needs at least one run");
    if (!runs) return bfail(PS_ERR_ARG, "null run array");
    if (nruns > (size_t)1 << 24) return bfail(PS_ERR_ARG, "at most 2^24 runs per batch");
    std::unordered_set<uintptr_t> states;
    for (size_t i = 0; i < nruns; ++i) {
        const ps_run_desc &r = runs[i];
        std::ostringstream os;
        os << "run " << i << ": ";
        if (r.n < 4 || r.n > 30) return bfail(PS_ERR_ARG, os.str() + "n must be in [4, 30]");
        if (r.count && (!r.x || !r.z || !r.phi)) return bfail(PS_ERR_ARG, os.str() + "null rotation array");
        if (need_ptrs) {
            if (!r.state) return bfail(PS_ERR_ARG, os.str() + "null state buffer");
            if ((((uintptr_t)r.state) | ((uintptr_t)r.psi0)) & 15)
                return bfail(PS_ERR_ARG, os.str() + "state buffers must be 16-byte aligned");
            if (!states.insert((uintptr_t)r.state).second)
                return bfail(PS_ERR_ARG, os.str() + "state buffer shared with another run");
        }
    }
    if (need_ptrs)
        for (size_t i = 0; i < nruns; ++i)
            if (runs[i].psi0 && states.count((uintptr_t)runs[i].psi0))
                return bfail(PS_ERR_ARG, "run " + std::to_string(i) + ": psi0 is the state buffer of a run");
    const int res = cfg.resident_bits < 0 ? 0 : cfg.resident_bits;
    const int single = cfg.single_bits < 0 ? 0 : cfg.single_bits;
    const int nlanes = grid / cfg.lane_size;

    L = Layout();
    L.runs.resize(nruns);
    L.work.resize(nruns);
    std::vector<Plan> plans(nruns);
    std::vector<int> kind(nruns), rc(nruns, PS_OK);
    std::vector<std::string> errs(nruns);
    for (size_t i = 0; i < nruns; ++i) {
        const int n = runs[i].n;
        kind[i] = n <= res ? -2 : (n <= single || nlanes == 0) ? -1 : 0;
    }
    // schedules, in parallel threads (each is independent host work)
    std::atomic<size_t> next{0};
    auto worker = [&]() {
        for (;;) {
            const size_t i = next.fetch_add(1);
            if (i >= nruns) return;
            const ps_run_desc &r = runs[i];
            Tuning t{};
            t.B = std::max(6, run_tile_bits(r.n, kind[i], cfg));
            t.G = kBatchG;
            t.max_window = batch_max_window(dtype);
            t.pair_single = 2;
            t.kernel_timing = 0;
            t.reg_groups = kBatchNG;  // recorded in the plan; the batched kernel fixes its own
            t.seg_bits = dtype == PS_C64 ? 4 : 3;
            t.tile_threads = 0;
            rc[i] = build_plan(r.n, dtype, r.x, r.z, r.phi, r.count, t, plans[i], &errs[i]);
        }
    };
    unsigned nth = std::max(1u, std::min(std::thread::hardware_concurrency(), 32u));
    nth = (unsigned)std::min<size_t>(nth, nruns);
    std::vector<std::thread> pool;
    for (unsigned k = 1; k < nth; ++k) pool.emplace_back(worker);
    worker();
    for (auto &th : pool) th.join();
    for (size_t i = 0; i < nruns; ++i)
        if (rc[i]) return bfail(rc[i], "run " + std::to_string(i) + ": " + errs[i]);

    // pack windows; every window is a tile pass (pair_single = 2)
    const size_t rec = dtype == PS_C64 ? kRecBytesC64 : kRecBytesC128;
    ps_batch_info &inf = L.info;
    for (size_t i = 0; i < nruns; ++i) {
        const Plan &p = plans[i];
        BatchRun &br = L.runs[i];
        br.n = runs[i].n;
        br.lane = kind[i];
        br.win_off = (uint32_t)L.wins.size();
        br.nwin = (uint32_t)p.win.size();
        if (p.B != run_tile_bits(br.n, kind[i], cfg) && !p.win.empty())
            return bfail(PS_ERR_ARG, "internal batch error (tile bits)");
        double pending = 1.0;
        for (size_t wi = 0; wi < p.win.size(); ++wi) {
            const WinDesc &w = p.win[wi];
            if (w.kind != 0) return bfail(PS_ERR_ARG, "internal batch error (pair window)");
            BatchWin bw{};
            bw.body = L.bodies.size();
            bw.B = w.c + w.d;
            bw.nsub = (int16_t)w.nsub;
            bw.nrot = (int16_t)w.nrot;
            // the same carried cos(phi) product as a single run, except that
            // the last window applies all of it
            pending *= w.kprod;
            const double dev = pending - 1.0;
            double kd = 0.0;
            if (wi + 1 == p.win.size() || std::fabs(dev) > (dtype == PS_C128 ? 0x1.0p-20 : 0x1.0p-16)) kd = dev;
            if (dtype == PS_C64) kd = (double)(float)kd;
            if (kd != 0.0) pending /= (1.0 + kd);
            bw.kdelta = kd;
            pack_window(p, w, L.bodies);
            L.wins.push_back(bw);
            L.smem = std::max(L.smem, (amp_bytes(dtype) << bw.B) + (size_t)batch_max_window(dtype) * rec);
        }
        const double N = std::ldexp(1.0, br.n);
        L.work[i] = N * (double)(br.nwin + 1);
        inf.rotations += runs[i].count;
        inf.windows += br.nwin;
        inf.amplitude_passes += N * (double)br.nwin;
        inf.amplitude_rotations += N * (double)runs[i].count;
        if (kind[i] == -2) {
            inf.resident_runs++;
            L.smem = std::max(L.smem, (amp_bytes(dtype) << br.n) + (size_t)batch_max_window(dtype) * rec);
        } else if (kind[i] == -1) {
            inf.single_runs++;
        } else {
            inf.lane_runs++;
        }
    }
    if (L.smem == 0) L.smem = (amp_bytes(dtype) << 4) + (size_t)batch_max_window(dtype) * rec;

    // lanes: longest first onto the least-loaded lane; each lane then runs
    // its runs longest first
    std::vector<int> lane_ix, single_ix;
    for (size_t i = 0; i < nruns; ++i) (kind[i] >= 0 ? lane_ix : single_ix).push_back((int)i);
    auto by_work = [&](int a, int b) { return L.work[a] != L.work[b] ? L.work[a] > L.work[b] : a < b; };
    std::sort(lane_ix.begin(), lane_ix.end(), by_work);
    std::sort(single_ix.begin(), single_ix.end(), by_work);
    L.nlanes = lane_ix.empty() ? 0 : nlanes;
    std::vector<std::vector<int>> lanes(L.nlanes);
    std::vector<double> load(L.nlanes, 0.0);
    using Item = std::pair<double, int>;  // (load, lane): lowest load, then lowest lane
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
    for (int l = 0; l < L.nlanes; ++l) pq.push({0.0, l});
    for (int i : lane_ix) {
        Item it = pq.top();
        pq.pop();
        lanes[it.second].push_back(i);
        L.runs[i].lane = it.second;
        load[it.second] += L.work[i];
        pq.push({load[it.second], it.second});
    }
    L.lane_off.assign(1, 0);
    for (int l = 0; l < L.nlanes; ++l) {
        for (int i : lanes[l]) L.lane_runs.push_back(i);
        L.lane_off.push_back((int)L.lane_runs.size());
    }
    L.single_order = single_ix;
    for (int i : single_ix) inf.single_work += L.work[i];
    for (double v : load) inf.max_lane_work = std::max(inf.max_lane_work, v);
    inf.runs = nruns;
    inf.body_bytes = L.bodies.size();
    inf.smem_bytes = L.smem;
    inf.lanes = L.nlanes;
    inf.lane_size = cfg.lane_size;
    inf.tile_bits = cfg.tile_bits;
    inf.resident_bits = cfg.resident_bits;
    inf.single_bits = cfg.single_bits;
    inf.grid = grid;
    if (cfg.withhold && (L.nlanes == 0 || cfg.lane_size < 2 || lanes[0].empty() || L.runs[lanes[0][0]].nwin == 0))
        return bfail(PS_ERR_ARG, "test_withhold needs lane_size >= 2 and a lane run with windows in lane 0");
    return PS_OK;
}

}  // namespace
}  // namespace ps

using namespace ps;

struct ps_batch {
    int dtype = 0;
    int device = 0;
    size_t nruns = 0;
    cudaStream_t stream = nullptr;
    BatchCfg cfg{};
    Layout L;
    BatchArgs args{};
    int grid = 0;
    // device memory: one block for the tables, one for the window bodies
    unsigned char *d_meta = nullptr;
    unsigned char *d_bodies = nullptr;
    void *d_ctrl = nullptr;     // status, queue, lane counters (cleared before every launch)
    size_t ctrl_bytes = 0;
    double *d_overlaps = nullptr;
    double *h_overlaps = nullptr;  // pinned
    int *h_status = nullptr;       // pinned
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool launched = false;
};

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int enqueue(ps_batch *b, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(b->d_ctrl, 0, b->ctrl_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_overlaps, 0, 2 * sizeof(double) * b->nruns, s);
    if (e != cudaSuccess) return cuda_bfail(e, "batch control reset");
    e = (cudaError_t)launch_batch(b->dtype, b->args, b->grid, b->L.smem, s);
    if (e != cudaSuccess) return cuda_bfail(e, "batch kernel launch (cooperative)");
    return PS_OK;
}

}  // namespace

extern "C" {

int ps_batch_describe(int dtype, const ps_run_desc *runs, size_t nruns, const ps_batch_config *cfg, int num_sms,
                      int ctas_per_sm, ps_batch_info *out, int *lane_of, int *tile_bits_of, uint64_t *windows_of) {
    BatchCfg c;
    if (int rc = resolve_cfg(dtype, cfg, c)) return rc;
    if (num_sms < 1 || ctas_per_sm < 1) return bfail(PS_ERR_ARG, "num_sms and ctas_per_sm must be >= 1");
    Layout L;
    if (int rc = build_layout(dtype, runs, nruns, c, num_sms * ctas_per_sm, false, L)) return rc;
    L.info.ctas_per_sm = ctas_per_sm;
    if (out) *out = L.info;
    for (size_t i = 0; i < nruns; ++i) {
        const BatchRun &r = L.runs[i];
        if (lane_of) lane_of[i] = r.lane;
        if (windows_of) windows_of[i] = r.nwin;
        if (tile_bits_of) tile_bits_of[i] = r.nwin ? L.wins[r.win_off].B : 0;
    }
    return PS_OK;
}

int ps_batch_create(int dtype, const ps_run_desc *runs, size_t nruns, const ps_batch_config *cfg, void *stream,
                    ps_batch **out) {
    if (!out) return bfail(PS_ERR_ARG, "null output pointer");
    *out = nullptr;
    BatchCfg c;
    if (int rc = resolve_cfg(dtype, cfg, c)) return rc;
    if (dtype != PS_C64 && dtype != PS_C128) return bfail(PS_ERR_ARG, "dtype must be PS_C64 or PS_C128");
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_bfail(e, "ps_batch_create: device query");
    int coop = 0;
    e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess) return cuda_bfail(e, "ps_batch_create: device query");
    if (!coop) return bfail(PS_ERR_UNSUPPORTED, "device does not support cooperative launches");

    // The grid depends on the shared memory, which the tile bits fix: no
    // tile exceeds 2^tile_bits amplitudes except a resident state.
    int max_res = 0, max_other = 0;
    if (runs)
        for (size_t i = 0; i < nruns; ++i) {
            if (runs[i].n <= c.resident_bits)
                max_res = std::max(max_res, runs[i].n);
            else
                max_other = std::max(max_other, std::min(runs[i].n, c.tile_bits));
        }
    const size_t smem = (amp_bytes(dtype) << std::max(4, std::max(max_res, max_other))) +
                        (size_t)batch_max_window(dtype) * (dtype == PS_C64 ? kRecBytesC64 : kRecBytesC128);
    e = (cudaError_t)batch_occupancy(dtype, smem, &occ);
    if (e != cudaSuccess) return cuda_bfail(e, "ps_batch_create: occupancy");
    if (occ < 1) return bfail(PS_ERR_UNSUPPORTED, "batched kernel does not fit on an SM with this shared memory");
    const int grid = occ * sms;

    ps_batch *b = new (std::nothrow) ps_batch();
    if (!b) return bfail(PS_ERR_OOM, "host allocation failed");
    b->dtype = dtype;
    b->device = dev;
    b->nruns = nruns;
    b->stream = (cudaStream_t)stream;
    b->cfg = c;
    b->grid = grid;
    if (int rc = build_layout(dtype, runs, nruns, c, grid, true, b->L)) {
        delete b;
        return rc;
    }
    Layout &L = b->L;
    L.smem = std::max(L.smem, smem);
    L.info.smem_bytes = L.smem;
    L.info.ctas_per_sm = occ;
    auto cleanup_fail = [&](int rc) {
        ps_batch_destroy(b);
        return rc;
    };

    // device tables in one block
    const size_t S = (size_t)c.lane_size;
    size_t off = 0;
    auto place = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    const size_t o_runs = place(sizeof(BatchRun) * nruns);
    const size_t o_wins = place(sizeof(BatchWin) * std::max<size_t>(1, L.wins.size()));
    const size_t o_states = place(sizeof(void *) * nruns);
    const size_t o_psi0 = place(sizeof(void *) * nruns);
    const size_t o_over = place(2 * sizeof(double) * nruns);
    const size_t o_part = place(2 * 2 * sizeof(double) * std::max<size_t>(1, (size_t)L.nlanes * S));
    const size_t o_lruns = place(sizeof(int) * std::max<size_t>(1, L.lane_runs.size()));
    const size_t o_loff = place(sizeof(int) * L.lane_off.size());
    const size_t o_single = place(sizeof(int) * std::max<size_t>(1, L.single_order.size()));
    // control: status, queue (one line), then the lanes' counters and generations
    b->ctrl_bytes = 128 + 2 * sizeof(unsigned) * kLaneStrideWords * std::max(1, L.nlanes);
    const size_t o_ctrl = place(b->ctrl_bytes);
    e = cudaMalloc((void **)&b->d_meta, off);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_bodies, std::max<size_t>(16, L.bodies.size()));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_overlaps, 2 * sizeof(double) * nruns);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&b->h_status, sizeof(int));
    if (e != cudaSuccess) return cleanup_fail(cuda_bfail(e, "ps_batch_create: allocation"));
    std::vector<unsigned char> host(off, 0);
    std::vector<void *> st(nruns), p0(nruns);
    for (size_t i = 0; i < nruns; ++i) {
        st[i] = runs[i].state;
        p0[i] = const_cast<void *>(runs[i].psi0);
    }
    std::memcpy(host.data() + o_runs, L.runs.data(), sizeof(BatchRun) * nruns);
    if (!L.wins.empty()) std::memcpy(host.data() + o_wins, L.wins.data(), sizeof(BatchWin) * L.wins.size());
    std::memcpy(host.data() + o_states, st.data(), sizeof(void *) * nruns);
    std::memcpy(host.data() + o_psi0, p0.data(), sizeof(void *) * nruns);
    if (!L.lane_runs.empty()) std::memcpy(host.data() + o_lruns, L.lane_runs.data(), sizeof(int) * L.lane_runs.size());
    std::memcpy(host.data() + o_loff, L.lane_off.data(), sizeof(int) * L.lane_off.size());
    if (!L.single_order.empty())
        std::memcpy(host.data() + o_single, L.single_order.data(), sizeof(int) * L.single_order.size());
    e = cudaMemcpy(b->d_meta, host.data(), off, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !L.bodies.empty())
        e = cudaMemcpy(b->d_bodies, L.bodies.data(), L.bodies.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cleanup_fail(cuda_bfail(e, "ps_batch_create: upload"));

    unsigned char *m = b->d_meta;
    b->d_ctrl = m + o_ctrl;
    b->d_overlaps = reinterpret_cast<double *>(m + o_over);
    BatchArgs &a = b->args;
    a.runs = reinterpret_cast<const BatchRun *>(m + o_runs);
    a.wins = reinterpret_cast<const BatchWin *>(m + o_wins);
    a.bodies = b->d_bodies;
    a.states = reinterpret_cast<void *const *>(m + o_states);
    a.psi0 = reinterpret_cast<const void *const *>(m + o_psi0);
    a.overlaps = b->d_overlaps;
    a.partials = reinterpret_cast<double *>(m + o_part);
    a.status = reinterpret_cast<int *>(m + o_ctrl);
    a.queue = reinterpret_cast<unsigned *>(m + o_ctrl + 64);
    a.lane_ctr = reinterpret_cast<unsigned *>(m + o_ctrl + 128);
    a.lane_gen = a.lane_ctr + (size_t)kLaneStrideWords * std::max(1, L.nlanes);
    a.lane_runs = reinterpret_cast<const int *>(m + o_lruns);
    a.lane_off = reinterpret_cast<const int *>(m + o_loff);
    a.single_order = reinterpret_cast<const int *>(m + o_single);
    a.nlanes = L.nlanes;
    a.lane_size = c.lane_size;
    a.nsingle = (int)L.single_order.size();
    a.withhold = c.withhold;
    a.budget_ns = (long long)c.wait_ms * 1000000ll;

    // capture the launch once; replays then cost one graph launch
    // (if this runtime cannot capture a cooperative launch, replays fall
    // back to plain launches and the info says graph = 0)
    if (c.use_graph == 1) {
        e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cleanup_fail(cuda_bfail(e, "ps_batch_create: capture stream"));
        e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int rc = enqueue(b, b->cap);
            cudaGraph_t g = nullptr;
            const cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
            if (rc == PS_OK && ee == cudaSuccess && g) {
                b->graph = g;
                if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) b->exec = nullptr;
            } else if (g) {
                cudaGraphDestroy(g);
            }
        }
        cudaGetLastError();
        set_error("");
        L.info.graph = b->exec ? 1 : 0;
    }
    *out = b;
    return PS_OK;
}

int ps_batch_launch(ps_batch *b) {
    if (!b) return bfail(PS_ERR_ARG, "null batch");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    int rc = PS_OK;
    if (b->exec) {
        const cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
        if (e != cudaSuccess) rc = cuda_bfail(e, "batch graph launch");
    } else {
        rc = enqueue(b, b->stream);
    }
    if (rc == PS_OK) b->launched = true;
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    return rc;
}

int ps_batch_wait(ps_batch *b, double *overlaps) {
    if (!b) return bfail(PS_ERR_ARG, "null batch");
    if (!b->launched) return bfail(PS_ERR_ARG, "ps_batch_wait before ps_batch_launch");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    cudaError_t e = cudaMemcpyAsync(b->h_status, b->args.status, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && overlaps)
        e = cudaMemcpyAsync(b->h_overlaps, b->d_overlaps, 2 * sizeof(double) * b->nruns, cudaMemcpyDeviceToHost,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_bfail(e, "ps_batch_wait");
    if (*b->h_status == PS_ERR_TIMEOUT) {
        std::ostringstream os;
        os << "batched launch: a lane barrier wait ran out after " << b->cfg.wait_ms
           << " ms; the states of this launch are undefined";
        return bfail(PS_ERR_TIMEOUT, os.str());
    }
    if (*b->h_status != PS_OK) return bfail(PS_ERR_CUDA, "batched launch reported an unknown status");
    if (overlaps) std::memcpy(overlaps, b->h_overlaps, 2 * sizeof(double) * b->nruns);
    return PS_OK;
}

int ps_batch_run(ps_batch *b, double *overlaps) {
    if (int rc = ps_batch_launch(b)) return rc;
    return ps_batch_wait(b, overlaps);
}

int ps_batch_get_info(const ps_batch *b, ps_batch_info *out) {
    if (!b || !out) return bfail(PS_ERR_ARG, "null argument");
    *out = b->L.info;
    return PS_OK;
}

void ps_batch_destroy(ps_batch *b) {
    if (!b) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != b->device) cudaSetDevice(b->device);
    if (b->launched) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->d_meta) cudaFree(b->d_meta);
    if (b->d_bodies) cudaFree(b->d_bodies);
    if (b->h_overlaps) cudaFreeHost(b->h_overlaps);
    if (b->h_status) cudaFreeHost(b->h_status);
    if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
    delete b;
}

}  // extern "C"
