// Batched persistent launch: many independent runs in one cooperative kernel.
//
// The paper runs its independent simulations (different Hamiltonians, times,
// step counts, random samples) as separate jobs, hundreds at a time (Methods,
// "Computational details"; Results, scaling runs).  On one GPU the same
// task-level parallelism becomes one persistent launch over all runs:
//   * lane runs: a lane of S co-resident CTAs takes its runs one after the
//     other; for every window it splits the 2^(n-B) tiles among its members
//     and meets at a lane barrier before the next window reads them;
//   * single runs: one CTA per run, taken from an atomic queue in longest-
//     first order once a CTA has finished its lane; a run whose whole state
//     fits in shared memory (2^n amplitudes) stays there for all its windows
//     and touches global memory only to read psi0 and to write the result.
// Every run ends with <psi0|psi> in FP64, summed in a fixed order.
// Every wait of one CTA for another is bounded by a %globaltimer budget:
// when it runs out the CTA records PS_ERR_TIMEOUT in the status word and
// returns, and every other waiting CTA returns once it sees the status.
#include <cuda_runtime.h>

#include "ps_tile.cuh"

namespace ps {

namespace {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_status(const int *p) { return *reinterpret_cast<const volatile int *>(p); }

// Barrier of one lane, called by thread 0 of each member after a
// __syncthreads (so the stores of all the CTA's threads precede its fence).
// Returns false when this CTA must stop: its wait ran out (the status
// becomes PS_ERR_TIMEOUT), another CTA reported a failure, or the test hook
// withholds this CTA's arrival.
__device__ bool lane_barrier0(const BatchArgs &A, int lane, bool withhold) {
    if (withhold) return false;
    unsigned *ctr = A.lane_ctr + (size_t)lane * kLaneStrideWords;
    unsigned *gen = A.lane_gen + (size_t)lane * kLaneStrideWords;
    bool ok = true;
    // the generation cannot move before this CTA arrives
    const unsigned g = ld_acquire(gen);
    __threadfence();
    const unsigned arrived = atomicAdd(ctr, 1u) + 1u;
    if (arrived == (unsigned)A.lane_size) {
        atomicExch(ctr, 0u);
        __threadfence();
        atomicAdd(gen, 1u);
    } else {
        const unsigned long long t0 = global_ns();
        while (ld_acquire(gen) == g) {
            if (ld_status(A.status) != PS_OK) {
                ok = false;
                break;
            }
            if (global_ns() - t0 > (unsigned long long)A.budget_ns) {
                atomicCAS(A.status, PS_OK, PS_ERR_TIMEOUT);
                ok = false;
                break;
            }
            __nanosleep(100);
        }
    }
    __threadfence();
    return ok;
}

// Copy a packed window (head, rounds, rotations) into the CTA's TileParams.
__device__ void load_window(TileParams &sP, const unsigned char *body, int nsub, int nrot) {
    __syncthreads();
    constexpr int kHeadWords = (int)(kWinHeadBytes / 8);
    const int sub_words = nsub * (int)(sizeof(TileSubP) / 4);
    const int sub_bytes = (nsub * (int)sizeof(TileSubP) + 7) & ~7;
    const int rot_words = nrot * (int)(sizeof(TileRotP) / 8);
    const uint64_t *h = reinterpret_cast<const uint64_t *>(body);
    const uint32_t *su = reinterpret_cast<const uint32_t *>(body + kWinHeadBytes);
    const uint64_t *ro = reinterpret_cast<const uint64_t *>(body + kWinHeadBytes + sub_bytes);
    uint64_t *dh = reinterpret_cast<uint64_t *>(&sP);
    uint32_t *dsu = reinterpret_cast<uint32_t *>(sP.sub);
    uint64_t *dro = reinterpret_cast<uint64_t *>(sP.rot);
    const int total = kHeadWords + sub_words + rot_words;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        if (i < kHeadWords)
            dh[i] = __ldg(h + i);
        else if (i < kHeadWords + sub_words)
            dsu[i - kHeadWords] = __ldg(su + (i - kHeadWords));
        else
            dro[i - kHeadWords - sub_words] = __ldg(ro + (i - kHeadWords - sub_words));
    }
    __syncthreads();
}

// FP64 sum of conj(psi0[k]) psi[k] over this CTA's range in a fixed order
// (thread-strided, then a fixed shuffle tree, then warps in order); the
// result is valid in thread 0.  With copy, the state out is first set to
// psi0 (a run without windows).  Otherwise, with out, psi is the CTA's
// shared-memory copy of the state and is written to out on the way.
template <typename C>
__device__ double2 cta_overlap(const C *psi0, const C *psi, C *out, size_t begin, size_t end, bool copy) {
    __shared__ double red[2][32];
    double re = 0.0, im = 0.0;
    for (size_t k = begin + threadIdx.x; k < end; k += blockDim.x) {
        const C a = __ldcg(psi0 + k);
        C b;
        if (copy) {
            b = a;
            out[k] = b;
        } else if (out) {
            b = psi[k];
            out[k] = b;
        } else {
            b = __ldcg(psi + k);
        }
        const double ar = (double)a.x, ai = (double)a.y, br = (double)b.x, bi = (double)b.y;
        re = fma(ar, br, fma(ai, bi, re));
        im = fma(ar, bi, fma(-ai, br, im));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = re;
        red[1][w] = im;
    }
    __syncthreads();
    double2 r = make_double2(0.0, 0.0);
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            r.x += red[0][i];
            r.y += red[1][i];
        }
    }
    return r;
}

// Write back a shared-memory-resident state without an overlap (psi0 absent).
template <typename C>
__device__ void cta_store(const C *tile, C *out, size_t count) {
    for (size_t k = threadIdx.x; k < count; k += blockDim.x) out[k] = tile[k];
}

// The CTA's copy of the current window.
__shared__ TileParams g_window;

// What the whole CTA does next, decided by thread 0.
enum : int { kOpDone = 0, kOpWindow, kOpTile, kOpTileGen, kOpLanePartial, kOpSingleEnd };

struct Item {
    int op;
    int r;          // run
    uint32_t h;     // kOpTile*: first tile, step and end of this CTA's tiles
    uint32_t hstep, ntile;
    int n;
    int flags;      // kOpTileGen: bit 0 load, bit 1 store to global; kOpSingleEnd: bit 0 resident
    int nwin;
    int nsub, nrot; // kOpWindow
    const void *src;
    void *dst;
    const unsigned char *body;
    double kdelta;
    uint64_t b0, b1;  // kOpLanePartial: slice of the state
    double *partial;  // kOpLanePartial: where thread 0 writes (re, im)
};

// Thread 0's position in its work: lane runs first, then single runs from
// the queue.
struct Cursor {
    int phase;  // 0 lane runs, 1 queue, 2 done
    int stage;  // 0 next run, 1 next window, 2 tiles of the window, 3 overlap partial, 4 overlap sum,
                // 5 end of window
    int lane, member, S, withhold;
    int q, q_end, r;
    int n, kind, nwin;
    uint32_t w, win_off, h, ntile;
    int B;
    double kdelta;
    const void *psi0;
    void *state;
};

// Advance the cursor to the next item of the CTA (thread 0 only; lane
// barriers wait here while the other threads wait at the CTA barrier).
template <int G, int NG, int LGT>
__device__ void next_item(const BatchArgs &A, Cursor &cu, Item &it) {
    for (;;) {
        if (cu.phase == 2) {
            it.op = kOpDone;
            return;
        }
        switch (cu.stage) {
        case 0: {  // next run
            if (cu.phase == 0) {
                if (cu.q >= cu.q_end) {
                    cu.phase = 1;
                    continue;
                }
                cu.r = A.lane_runs[cu.q];
            } else {
                if (ld_status(A.status) != PS_OK) {
                    cu.phase = 2;
                    continue;
                }
                const unsigned slot = atomicAdd(A.queue, 1u);
                if (slot >= (unsigned)A.nsingle) {
                    cu.phase = 2;
                    continue;
                }
                cu.r = A.single_order[slot];
            }
            const BatchRun run = A.runs[cu.r];
            cu.n = run.n;
            cu.kind = run.lane;
            cu.nwin = (int)run.nwin;
            cu.win_off = run.win_off;
            cu.state = A.states[cu.r];
            cu.psi0 = A.psi0[cu.r];
            cu.w = 0;
            cu.stage = 1;
            continue;
        }
        case 1: {  // next window
            if (cu.w >= (uint32_t)cu.nwin) {
                if (cu.phase == 0) {
                    cu.stage = 3;
                    continue;
                }
                it.op = kOpSingleEnd;
                it.r = cu.r;
                it.n = cu.n;
                it.nwin = cu.nwin;
                it.flags = cu.kind == -2 ? 1 : 0;
                it.src = cu.psi0;
                it.dst = cu.state;
                cu.stage = 0;
                return;
            }
            const BatchWin bw = A.wins[cu.win_off + cu.w];
            cu.kdelta = bw.kdelta;
            cu.B = bw.B;
            cu.ntile = 1u << (cu.n - bw.B);
            cu.h = cu.phase == 0 ? (uint32_t)cu.member : 0u;
            cu.stage = 2;
            it.op = kOpWindow;
            it.body = A.bodies + bw.body;
            it.nsub = bw.nsub;
            it.nrot = bw.nrot;
            return;
        }
        case 2: {  // this CTA's tiles of the window, all in one item
            const bool resident = cu.kind == -2;
            // a full block of register groups: 2^(B - G) / NG >= 2^LGT threads
            const bool full = !resident && cu.B - G - (NG == 4 ? 2 : NG == 2 ? 1 : 0) >= LGT;
            it.op = full ? kOpTile : kOpTileGen;
            it.h = cu.h;
            it.hstep = cu.phase == 0 ? (uint32_t)cu.S : 1u;
            it.ntile = cu.ntile;
            it.n = cu.n;
            it.kdelta = cu.kdelta;
            it.src = (cu.w == 0 && cu.psi0) ? cu.psi0 : cu.state;
            it.dst = cu.state;
            it.flags = ((!resident || cu.w == 0) ? 1 : 0) | (resident ? 0 : 2);
            cu.stage = 5;
            return;
        }
        case 5: {  // end of window: lane barrier before the next window reads
            if (cu.phase == 0 && !lane_barrier0(A, cu.lane, cu.withhold != 0)) {
                cu.phase = 2;
                continue;
            }
            cu.w++;
            cu.stage = 1;
            continue;
        }
        case 3: {  // overlap: this member's slice
            if (!cu.psi0) {
                cu.q++;
                cu.stage = 0;
                continue;
            }
            const uint64_t N = 1ull << cu.n;
            const uint64_t per = (N + cu.S - 1) / cu.S;
            it.op = kOpLanePartial;
            it.r = cu.r;
            it.nwin = cu.nwin;
            it.src = cu.psi0;
            it.dst = cu.state;
            it.b0 = min(N, per * (uint64_t)cu.member);
            it.b1 = min(N, it.b0 + per);
            // two buffers: a member may start the next run's partial while
            // member 0 still sums this one's
            it.partial = A.partials + 2 * ((size_t)(cu.q & 1) * A.nlanes * cu.S + (size_t)cu.lane * cu.S + cu.member);
            cu.stage = 4;
            return;
        }
        case 4: {  // overlap: member 0 sums the partials in member order
            if (!lane_barrier0(A, cu.lane, cu.withhold != 0)) {
                cu.phase = 2;
                continue;
            }
            if (cu.member == 0) {
                const double *pp = A.partials + 2 * ((size_t)(cu.q & 1) * A.nlanes * cu.S + (size_t)cu.lane * cu.S);
                double re = 0.0, im = 0.0;
                for (int m = 0; m < cu.S; ++m) {
                    re += __ldcg(pp + 2 * m);
                    im += __ldcg(pp + 2 * m + 1);
                }
                A.overlaps[2 * cu.r] = re;
                A.overlaps[2 * cu.r + 1] = im;
            }
            cu.q++;
            cu.stage = 0;
            continue;
        }
        default:
            cu.phase = 2;
            continue;
        }
    }
}

// Persistent CTA: thread 0 picks the next item, the whole CTA executes it.
// No loop state lives in registers across a tile pass (it is all in the
// shared cursor), so each pass has the single-window kernel's register
// budget to itself.
template <typename R, int G, int NG>
__global__ void __launch_bounds__(batch_threads<R>(), 3) k_batch(const __grid_constant__ BatchArgs A) {
    using C = typename CT<R>::T;
    constexpr int LGT = batch_threads<R>() == 128 ? 7 : 8;
    static_assert(batch_threads<R>() == (1 << LGT), "128 or 256 threads");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Cursor cu;
    __shared__ Item it;
    if (threadIdx.x == 0) {
        const int S = A.lane_size;
        cu.S = S;
        cu.lane = (int)blockIdx.x / S;
        cu.member = (int)blockIdx.x % S;
        cu.withhold = (A.withhold && cu.lane == 0 && cu.member == S - 1 && S > 1) ? 1 : 0;
        cu.stage = 0;
        if (cu.lane < A.nlanes) {
            cu.phase = 0;
            cu.q = A.lane_off[cu.lane];
            cu.q_end = A.lane_off[cu.lane + 1];
        } else {
            cu.phase = 1;
        }
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) next_item<G, NG, LGT>(A, cu, it);
        __syncthreads();
        const int op = it.op;
        if (op == kOpDone) break;
        if (op == kOpTile) {
            // only h stays in a register across a pass; the rest is re-read
            // from shared memory after the pass's barriers
            for (uint32_t h = it.h; h < it.ntile; h += it.hstep)
                tile_pass<R, G, NG, false>(reinterpret_cast<const C *>(it.src), reinterpret_cast<C *>(it.dst),
                                           g_window, h, it.n, (R)it.kdelta, true, true);
        } else if (op == kOpTileGen) {
            for (uint32_t h = it.h; h < it.ntile; h += it.hstep)
                tile_pass<R, G, NG, true>(reinterpret_cast<const C *>(it.src), reinterpret_cast<C *>(it.dst),
                                          g_window, h, it.n, (R)it.kdelta, (it.flags & 1) != 0, (it.flags & 2) != 0);
        } else if (op == kOpWindow) {
            load_window(g_window, it.body, it.nsub, it.nrot);
        } else if (op == kOpLanePartial) {
            const bool copy = it.nwin == 0;
            C *state = reinterpret_cast<C *>(it.dst);
            const double2 p = cta_overlap<C>(reinterpret_cast<const C *>(it.src), state, copy ? state : nullptr,
                                             it.b0, it.b1, copy);
            if (threadIdx.x == 0) {
                it.partial[0] = p.x;
                it.partial[1] = p.y;
            }
        } else if (op == kOpSingleEnd) {
            const C *psi0 = reinterpret_cast<const C *>(it.src);
            C *state = reinterpret_cast<C *>(it.dst);
            const size_t N = (size_t)1 << it.n;
            const C *tile = reinterpret_cast<const C *>(smem);
            const bool resident = (it.flags & 1) && it.nwin > 0;
            if (psi0) {
                // a resident run leaves shared memory on the way
                const double2 p = cta_overlap<C>(psi0, resident ? tile : state,
                                                 (resident || it.nwin == 0) ? state : nullptr, 0, N, it.nwin == 0);
                if (threadIdx.x == 0) {
                    A.overlaps[2 * it.r] = p.x;
                    A.overlaps[2 * it.r + 1] = p.y;
                }
            } else if (resident) {
                cta_store<C>(tile, state, N);
            }
        }
    }
}

template <typename R>
void *batch_kernel() {
    return reinterpret_cast<void *>(&k_batch<R, kBatchG, kBatchNG>);
}

}  // namespace

int batch_occupancy(int dtype, size_t smem_bytes, int *blocks_per_sm) {
    void *fn = dtype == PS_C64 ? batch_kernel<float>() : batch_kernel<double>();
    // the limit is an upper bound for every batch; each launch asks for what it uses
    constexpr int kBatchSmemLimit = 200 * 1024;
    if (smem_bytes > (size_t)kBatchSmemLimit) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmemLimit);
    const int threads = dtype == PS_C64 ? batch_threads<float>() : batch_threads<double>();
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, threads, smem_bytes);
    return (int)e;
}

int launch_batch(int dtype, const BatchArgs &a, int grid, size_t smem_bytes, void *stream) {
    void *fn = dtype == PS_C64 ? batch_kernel<float>() : batch_kernel<double>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)(dtype == PS_C64 ? batch_threads<float>() : batch_threads<double>()));
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {const_cast<BatchArgs *>(&a)};
    return (int)cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace ps
