// Data movement of the qubit-swap exchange (include/ps.h, ps_shard_pack /
// ps_shard_unpack).  Swapping k rank positions with the k slab positions of
// lmask (paired in ascending order) sends part j of every slab -- the
// amplitudes whose bits at lmask spell j, in the order of their other bits --
// to the rank whose swapped bits spell j; the part received from the rank
// whose swapped bits spell j' lands at the slab indices with j' at lmask.
// Packed index i = j 2^(s-k) + c names amplitude c of part j; both kernels
// move any range of packed indices (a whole slab, one part, or a chunk of
// one), reading and writing every amplitude of the range once.
#include <cuda_runtime.h>

#include "ps_device.cuh"
#include "ps_internal.h"

namespace ps {
namespace {

constexpr int kShardThreads = 256;

struct SwapPositions {
    int k;
    int p[20];  // ascending slab positions
};

__device__ __forceinline__ uint64_t insert_bits(uint64_t c, uint32_t j, const SwapPositions &sp) {
    for (int t = 0; t < sp.k; ++t) {
        const int p = sp.p[t];
        c = ((c >> p) << (p + 1)) | (c & ((1ull << p) - 1)) | ((uint64_t)((j >> t) & 1u) << p);
    }
    return c;
}

// PACK: out[j 2^(s-k) + c] = slab[insert(c, j)];  else slab[insert(c, j)] = in[j 2^(s-k) + c]
template <typename C, bool PACK>
__global__ void __launch_bounds__(kShardThreads) k_shard_move(const C *__restrict__ src, C *__restrict__ dst, int s,
                                                              const SwapPositions sp, uint64_t first,
                                                              uint64_t count) {
    const int lc = s - sp.k;
    const uint64_t cmask = (1ull << lc) - 1;
    for (uint64_t r = (uint64_t)blockIdx.x * kShardThreads + threadIdx.x; r < count;
         r += (uint64_t)gridDim.x * kShardThreads) {
        const uint64_t i = first + r;
        const uint64_t at = insert_bits(i & cmask, (uint32_t)(i >> lc), sp);
        if (PACK)
            dst[r] = src[at];
        else
            dst[at] = src[r];
    }
}

int shard_move(bool pack, int s, int dtype, uint64_t lmask, uint64_t first, uint64_t count, const void *src,
               void *dst, void *stream) {
    SwapPositions sp{};
    sp.k = 0;
    for (int p = 0; p < 64; ++p)
        if ((lmask >> p) & 1) sp.p[sp.k++] = p;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t blocks = (count + kShardThreads - 1) / kShardThreads;
    if (blocks == 0) return 0;
    const uint64_t cap = (uint64_t)(sms > 0 ? sms : 1) * 8;
    if (blocks > cap) blocks = cap;
    cudaStream_t st = (cudaStream_t)stream;
    if (dtype == PS_C64) {
        if (pack)
            k_shard_move<float2, true><<<(unsigned)blocks, kShardThreads, 0, st>>>((const float2 *)src, (float2 *)dst, s, sp, first, count);
        else
            k_shard_move<float2, false><<<(unsigned)blocks, kShardThreads, 0, st>>>((const float2 *)src, (float2 *)dst, s, sp, first, count);
    } else {
        if (pack)
            k_shard_move<double2, true><<<(unsigned)blocks, kShardThreads, 0, st>>>((const double2 *)src, (double2 *)dst, s, sp, first, count);
        else
            k_shard_move<double2, false><<<(unsigned)blocks, kShardThreads, 0, st>>>((const double2 *)src, (double2 *)dst, s, sp, first, count);
    }
    return (int)cudaGetLastError();
}

int check_move(int s, int dtype, uint64_t lmask, uint64_t first, uint64_t count, const void *a, const void *b) {
    if (dtype != PS_C64 && dtype != PS_C128) {
        set_error("dtype must be PS_C64 or PS_C128");
        return PS_ERR_ARG;
    }
    if (s < 1 || s > kMaxN) {
        set_error("s must be in [1, 40]");
        return PS_ERR_ARG;
    }
    const int k = __builtin_popcountll(lmask);
    if (k < 1 || k > 20 || k > s || (lmask >> s)) {
        set_error("lmask must name 1..min(20, s) slab positions below s");
        return PS_ERR_ARG;
    }
    if (!a || !b || a == b) {
        set_error("source and destination must be distinct device buffers");
        return PS_ERR_ARG;
    }
    if (first > (1ull << s) || count > (1ull << s) - first) {
        set_error("packed range outside the slab's 2^s amplitudes");
        return PS_ERR_ARG;
    }
    return PS_OK;
}

}  // namespace
}  // namespace ps

extern "C" int ps_shard_pack(int s, int dtype, uint64_t lmask, uint64_t first, uint64_t count, const void *slab_dev,
                             void *out_dev, void *stream) {
    using namespace ps;
    if (int rc = check_move(s, dtype, lmask, first, count, slab_dev, out_dev)) return rc;
    const int e = shard_move(true, s, dtype, lmask, first, count, slab_dev, out_dev, stream);
    if (e) {
        set_error(std::string("shard pack kernel: ") + cudaGetErrorString((cudaError_t)e));
        return PS_ERR_CUDA;
    }
    return PS_OK;
}

extern "C" int ps_shard_unpack(int s, int dtype, uint64_t lmask, uint64_t first, uint64_t count, const void *in_dev,
                               void *slab_dev, void *stream) {
    using namespace ps;
    if (int rc = check_move(s, dtype, lmask, first, count, in_dev, slab_dev)) return rc;
    const int e = shard_move(false, s, dtype, lmask, first, count, in_dev, slab_dev, stream);
    if (e) {
        set_error(std::string("shard unpack kernel: ") + cudaGetErrorString((cudaError_t)e));
        return PS_ERR_CUDA;
    }
    return PS_OK;
}
