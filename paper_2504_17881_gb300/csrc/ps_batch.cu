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

// Barrier of one lane.  Returns false when this CTA must stop: its wait ran
// out (the status becomes PS_ERR_TIMEOUT), another CTA reported a failure,
// or the test hook withholds this CTA's arrival.
__device__ bool lane_barrier(const BatchArgs &A, int lane, bool withhold) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (withhold) {
            ok = 0;
        } else {
            unsigned *ctr = A.lane_ctr + (size_t)lane * kLaneStrideWords;
            unsigned *gen = A.lane_gen + (size_t)lane * kLaneStrideWords;
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
                        ok = 0;
                        break;
                    }
                    if (global_ns() - t0 > (unsigned long long)A.budget_ns) {
                        atomicCAS(A.status, PS_OK, PS_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(100);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
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

// All windows of run r on this CTA: tiles member, member + S, ... of every
// window, then the lane barrier (lane >= 0).  A resident run (lane -2) has
// one tile per window, the whole state, which stays in shared memory: only
// the first window loads it, no window stores it.  One call site of the tile
// pass for every kind of run keeps the kernel's code (and its registers) to
// one copy of the pass.  Returns false when the CTA must stop.
template <typename R, int G, int NG>
__device__ __noinline__ bool run_windows(const BatchArgs &A, int r, int lane, int member, int S, bool withhold) {
    using C = typename CT<R>::T;
    const BatchRun run = A.runs[r];
    C *state = reinterpret_cast<C *>(A.states[r]);
    const C *psi0 = reinterpret_cast<const C *>(A.psi0[r]);
    const bool resident = run.lane == -2;
    for (uint32_t w = 0; w < run.nwin; ++w) {
        const BatchWin bw = A.wins[run.win_off + w];
        load_window(g_window, A.bodies + bw.body, bw.nsub, bw.nrot);
        const C *src = (w == 0 && psi0) ? psi0 : state;
        const uint32_t ntile = 1u << (run.n - bw.B);
        for (uint32_t h = (uint32_t)member; h < ntile; h += (uint32_t)S)
            tile_pass<R, G, NG, true>(src, state, g_window, h, run.n, (R)bw.kdelta, !resident || w == 0, !resident);
        if (lane >= 0 && !lane_barrier(A, lane, withhold)) return false;
    }
    return true;
}

template <typename R, int G, int NG>
__global__ void __launch_bounds__(kBatchThreads, tile_min_blocks<R, G, NG>()) k_batch(const __grid_constant__ BatchArgs A) {
    using C = typename CT<R>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned s_slot;
    const int S = A.lane_size;
    const int lane = (int)blockIdx.x / S, member = (int)blockIdx.x % S;

    // ---------------------------------------------------------- lane runs
    if (lane < A.nlanes) {
        const bool withhold = A.withhold && lane == 0 && member == S - 1 && S > 1;
        for (int q = A.lane_off[lane]; q < A.lane_off[lane + 1]; ++q) {
            const int r = A.lane_runs[q];
            if (!run_windows<R, G, NG>(A, r, lane, member, S, withhold)) return;
            const C *psi0 = reinterpret_cast<const C *>(A.psi0[r]);
            if (!psi0) continue;
            C *state = reinterpret_cast<C *>(A.states[r]);
            const BatchRun run = A.runs[r];
            // member m sums its slice; partials alternate between two buffers
            // so a member may start the next run's epilogue while member 0
            // still reads this one's
            const size_t N = (size_t)1 << run.n;
            const size_t per = (N + S - 1) / S;
            const size_t b0 = min(N, per * member), b1 = min(N, b0 + per);
            const double2 p = cta_overlap<C>(psi0, state, run.nwin == 0 ? state : nullptr, b0, b1, run.nwin == 0);
            double *part = A.partials + 2 * ((size_t)(q & 1) * A.nlanes * S + (size_t)lane * S + member);
            if (threadIdx.x == 0) {
                part[0] = p.x;
                part[1] = p.y;
            }
            if (!lane_barrier(A, lane, withhold)) return;
            if (member == 0 && threadIdx.x == 0) {
                const double *pp = A.partials + 2 * ((size_t)(q & 1) * A.nlanes * S + (size_t)lane * S);
                double re = 0.0, im = 0.0;
                for (int m = 0; m < S; ++m) {
                    re += __ldcg(pp + 2 * m);
                    im += __ldcg(pp + 2 * m + 1);
                }
                A.overlaps[2 * r] = re;
                A.overlaps[2 * r + 1] = im;
            }
        }
    }

    // --------------------------------------------------------- single runs
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_slot = atomicAdd(A.queue, 1u);
        __syncthreads();
        const unsigned slot = s_slot;
        if (slot >= (unsigned)A.nsingle) break;
        if (ld_status(A.status) != PS_OK) break;
        const int r = A.single_order[slot];
        run_windows<R, G, NG>(A, r, -1, 0, 1, false);
        __syncthreads();
        const BatchRun run = A.runs[r];
        C *state = reinterpret_cast<C *>(A.states[r]);
        const C *psi0 = reinterpret_cast<const C *>(A.psi0[r]);
        const size_t N = (size_t)1 << run.n;
        const C *tile = reinterpret_cast<const C *>(smem);
        const bool resident = run.lane == -2 && run.nwin > 0;
        if (psi0) {
            // a resident run leaves shared memory on the way
            const double2 p = cta_overlap<C>(psi0, resident ? tile : state,
                                             (resident || run.nwin == 0) ? state : nullptr, 0, N, run.nwin == 0);
            if (threadIdx.x == 0) {
                A.overlaps[2 * r] = p.x;
                A.overlaps[2 * r + 1] = p.y;
            }
        } else if (resident) {
            cta_store<C>(tile, state, N);
        }
    }
}

template <typename R>
void *batch_kernel() {
    return reinterpret_cast<void *>(&k_batch<R, kBatchG, 2>);
}

}  // namespace

int batch_occupancy(int dtype, size_t smem_bytes, int *blocks_per_sm) {
    void *fn = dtype == PS_C64 ? batch_kernel<float>() : batch_kernel<double>();
    // the limit is an upper bound for every batch; each launch asks for what it uses
    constexpr int kBatchSmemLimit = 200 * 1024;
    if (smem_bytes > (size_t)kBatchSmemLimit) return (int)cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchSmemLimit);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kBatchThreads, smem_bytes);
    return (int)e;
}

int launch_batch(int dtype, const BatchArgs &a, int grid, size_t smem_bytes, void *stream) {
    void *fn = dtype == PS_C64 ? batch_kernel<float>() : batch_kernel<double>();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBatchThreads);
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
