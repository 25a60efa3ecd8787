// FP32 kernels of the step-count predictor: a multilayer perceptron with three
// tanh hidden layers of 128 units and a linear scalar output, trained with
// mean-squared error and Adam.  See ps_mlp_host.cpp for the object around
// them and include/ps.h for the parameter layout.
//
// The network is small (34.6k parameters) and its cost is negligible next
// to generating its training data, so the kernels aim for simple,
// deterministic code: weights staged in shared memory, every sum in a fixed
// order (no atomics), FP32 arithmetic with the library's tanhf.
#include <cuda_runtime.h>

#include "ps_internal.h"

namespace ps {

namespace {

constexpr int W = kMlpWidth;        // 128 hidden units
constexpr int ROWS = 32;            // rows per CTA in forward / backward
constexpr int THREADS = 256;
constexpr int WS_STRIDE = W + 1;    // padded shared-memory row of a staged weight matrix

struct Offsets {
    int W1, b1, W2, b2, W3, b3, wo, bo, total;
};

__host__ __device__ inline Offsets offsets(int n_in) {
    Offsets o;
    o.W1 = 0;
    o.b1 = o.W1 + W * n_in;
    o.W2 = o.b1 + W;
    o.b2 = o.W2 + W * W;
    o.W3 = o.b2 + W;
    o.b3 = o.W3 + W * W;
    o.wo = o.b3 + W;
    o.bo = o.wo + W;
    o.total = o.bo + 1;
    return o;
}

// x_std = (x - mu) * inv_sigma per feature; y likewise (when given).
__global__ void k_mlp_standardize(const float *__restrict__ x, const float *__restrict__ y, int rows, int n_in,
                                  MlpNorm nm, float *__restrict__ xs, float *__restrict__ ys) {
    const int total = rows * n_in;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int f = e % n_in;
        xs[e] = (x[e] - nm.mu[f]) * nm.inv_sigma[f];
    }
    if (y)
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows; e += gridDim.x * blockDim.x)
            ys[e] = (y[e] - nm.y_mu) * nm.y_inv_sigma;
}

// Stage W (out-major, n_out x n_in in global memory) transposed into
// ws[i * WS_STRIDE + o], so a thread per output o reads consecutive banks.
__device__ void stage_transposed(const float *__restrict__ Wg, int n_in, float *ws) {
    for (int e = threadIdx.x; e < W * n_in; e += blockDim.x) {
        const int o = e / n_in, i = e % n_in;
        ws[i * WS_STRIDE + o] = Wg[e];
    }
}

// Stage W as stored (out-major): ws[o * WS_STRIDE + i], a thread per input i.
__device__ void stage_direct(const float *__restrict__ Wg, float *ws) {
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
        const int o = e / W, i = e % W;
        ws[o * WS_STRIDE + i] = Wg[e];
    }
}

// Forward pass of ROWS rows per CTA.  Rows r of the call are rows idx[r] of
// xs (or r itself without idx).  acts (3 x rows x W, optional) receives the
// hidden activations; out the scalar output, de-standardised when denorm.
__global__ void __launch_bounds__(THREADS) k_mlp_forward(const float *__restrict__ P, const float *__restrict__ xs,
                                                         const int *__restrict__ idx, int rows, int n_in,
                                                         float *__restrict__ acts, float *__restrict__ out,
                                                         int denorm, float y_mu, float y_sigma) {
    extern __shared__ __align__(16) float sh[];
    float *ws = sh;                          // W x WS_STRIDE
    float *ha = ws + W * WS_STRIDE;          // ROWS x W
    float *hb = ha + ROWS * W;               // ROWS x W
    const Offsets of = offsets(n_in);
    const int row0 = blockIdx.x * ROWS;
    const int nr = min(ROWS, rows - row0);
    const int o = threadIdx.x & (W - 1);
    const int rg = threadIdx.x >> 7;         // two row groups of 16
    // inputs
    for (int e = threadIdx.x; e < ROWS * n_in; e += blockDim.x) {
        const int r = e / n_in, i = e % n_in;
        float v = 0.f;
        if (r < nr) {
            const int src = idx ? idx[row0 + r] : row0 + r;
            v = xs[(size_t)src * n_in + i];
        }
        ha[r * W + i] = v;
    }
    stage_transposed(P + of.W1, n_in, ws);
    __syncthreads();
    const int K[3] = {n_in, W, W};
    const int offW[3] = {of.W1, of.W2, of.W3};
    const int offb[3] = {of.b1, of.b2, of.b3};
    float *hin = ha, *hout = hb;
    for (int layer = 0; layer < 3; ++layer) {
        if (layer > 0) {
            __syncthreads();
            stage_transposed(P + offW[layer], W, ws);
            __syncthreads();
        }
        float acc[16];
        const float b = P[offb[layer] + o];
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) acc[rr] = b;
        for (int i = 0; i < K[layer]; ++i) {
            const float w = ws[i * WS_STRIDE + o];
#pragma unroll
            for (int rr = 0; rr < 16; ++rr) acc[rr] = fmaf(w, hin[(rg * 16 + rr) * W + i], acc[rr]);
        }
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
            const int r = rg * 16 + rr;
            const float h = tanhf(acc[rr]);
            hout[r * W + o] = h;
            if (acts && r < nr) acts[((size_t)layer * rows + row0 + r) * W + o] = h;
        }
        float *t = hin;
        hin = hout;
        hout = t;
    }
    __syncthreads();
    // output: warp w handles rows 4w .. 4w+3; fixed-order lane sums
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float bo = P[of.bo];
    for (int k = 0; k < ROWS / 8; ++k) {
        const int r = warp * (ROWS / 8) + k;
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < W / 32; ++j) s = fmaf(P[of.wo + lane + 32 * j], hin[r * W + lane + 32 * j], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0 && r < nr) {
            const float y = s + bo;
            out[row0 + r] = denorm ? fmaf(y_sigma, y, y_mu) : y;
        }
    }
}

// Backward pass of ROWS rows per CTA for the loss (1/B) sum (out - t)^2.
// deltas: three blocks of rows x W (dL/d pre-activation of hidden layers 1..3)
// then rows values of dL/d out.  loss_part[blockIdx.x] = the CTA's sum of
// squared errors.
__global__ void __launch_bounds__(THREADS) k_mlp_backward(const float *__restrict__ P, const float *__restrict__ ts,
                                                          const int *__restrict__ idx, int rows, int n_in, float inv_B,
                                                          const float *__restrict__ acts,
                                                          const float *__restrict__ out, float *__restrict__ deltas,
                                                          float *__restrict__ loss_part) {
    extern __shared__ __align__(16) float sh[];
    float *ws = sh;
    float *da = ws + W * WS_STRIDE;
    float *db = da + ROWS * W;
    __shared__ float dout[ROWS];
    __shared__ float sq[ROWS];
    const Offsets of = offsets(n_in);
    const int row0 = blockIdx.x * ROWS;
    const int nr = min(ROWS, rows - row0);
    const int c = threadIdx.x & (W - 1);
    const int rg = threadIdx.x >> 7;
    if (threadIdx.x < ROWS) {
        const int r = threadIdx.x;
        float d = 0.f, e2 = 0.f;
        if (r < nr) {
            const int src = idx ? idx[row0 + r] : row0 + r;
            const float e = out[row0 + r] - ts[src];
            d = 2.f * e * inv_B;
            e2 = e * e;
            deltas[(size_t)3 * rows * W + row0 + r] = d;
        }
        dout[r] = d;
        sq[r] = e2;
    }
    stage_direct(P + of.W3, ws);
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int r = 0; r < ROWS; ++r) s += sq[r];
        loss_part[blockIdx.x] = s;
    }
    // delta of hidden layer 3
    const float wo = P[of.wo + c];
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
        const int r = rg * 16 + rr;
        float d = 0.f;
        if (r < nr) {
            const float h = acts[((size_t)2 * rows + row0 + r) * W + c];
            d = dout[r] * wo * (1.f - h * h);
            deltas[((size_t)2 * rows + row0 + r) * W + c] = d;
        }
        da[r * W + c] = d;
    }
    __syncthreads();
    // deltas of hidden layers 2 and 1: (delta_next W_next)_i (1 - h_i^2)
    float *din = da, *dnext = db;
    for (int layer = 1; layer >= 0; --layer) {
        if (layer == 0) {
            __syncthreads();
            stage_direct(P + of.W2, ws);
            __syncthreads();
        }
        float acc[16];
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) acc[rr] = 0.f;
        for (int oo = 0; oo < W; ++oo) {
            const float w = ws[oo * WS_STRIDE + c];
#pragma unroll
            for (int rr = 0; rr < 16; ++rr) acc[rr] = fmaf(din[(rg * 16 + rr) * W + oo], w, acc[rr]);
        }
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
            const int r = rg * 16 + rr;
            float d = 0.f;
            if (r < nr) {
                const float h = acts[((size_t)layer * rows + row0 + r) * W + c];
                d = acc[rr] * (1.f - h * h);
                deltas[((size_t)layer * rows + row0 + r) * W + c] = d;
            }
            dnext[r * W + c] = d;
        }
        float *t = din;
        din = dnext;
        dnext = t;
    }
}

// Weight gradients: dW[o][i] = sum_rows delta[row][o] in[row][i] and the bias
// as input column i = K (value 1), summed over the rows in order.  One CTA
// per 32 x 32 tile of (outputs, inputs + 1) of one layer; tiles of the four
// layers are numbered consecutively (see k_mlp_wgrad_tiles).
__global__ void __launch_bounds__(THREADS) k_mlp_wgrad(const float *__restrict__ xs, const int *__restrict__ idx,
                                                       int rows, int n_in, const float *__restrict__ acts,
                                                       const float *__restrict__ deltas, float *__restrict__ G) {
    __shared__ float sd[32][33];
    __shared__ float si[32][33];
    const Offsets of = offsets(n_in);
    // tiles: layer 1: 4 (o) x 1; layers 2, 3: 4 x 5 each; output: 1 x 5
    int t = blockIdx.x;
    int layer, to, ti, K, n_out;
    if (t < 4) {
        layer = 0; to = t; ti = 0; K = n_in; n_out = W;
    } else if (t < 24) {
        layer = 1; t -= 4; to = t / 5; ti = t % 5; K = W; n_out = W;
    } else if (t < 44) {
        layer = 2; t -= 24; to = t / 5; ti = t % 5; K = W; n_out = W;
    } else {
        layer = 3; t -= 44; to = 0; ti = t; K = W; n_out = 1;
    }
    const float *dsrc = deltas + (size_t)layer * rows * W;  // layer 3: the dL/d out values
    const int dstride = layer == 3 ? 1 : W;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty in 0..7: four outputs each
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int r0 = 0; r0 < rows; r0 += 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
            const int rr = e >> 5, cc = e & 31;
            const int r = r0 + rr;
            const int oo = to * 32 + cc, ii = ti * 32 + cc;
            float dv = 0.f, iv = 0.f;
            if (r < rows) {
                if (oo < n_out) dv = dsrc[(size_t)r * dstride + oo];
                if (ii < K) {
                    if (layer == 0) {
                        const int src = idx ? idx[r] : r;
                        iv = xs[(size_t)src * n_in + ii];
                    } else {
                        iv = acts[((size_t)(layer - 1) * rows + r) * W + ii];
                    }
                } else if (ii == K) {
                    iv = 1.f;
                }
            }
            sd[rr][cc] = dv;
            si[rr][cc] = iv;
        }
        __syncthreads();
        for (int rr = 0; rr < 32; ++rr) {
            const float x = si[rr][tx];
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] = fmaf(sd[rr][ty * 4 + k], x, acc[k]);
        }
    }
    const int ii = ti * 32 + tx;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int oo = to * 32 + ty * 4 + k;
        if (oo >= n_out || ii > K) continue;
        int dst;
        if (layer == 3)
            dst = ii < K ? of.wo + ii : of.bo;
        else {
            const int ow = layer == 0 ? of.W1 : (layer == 1 ? of.W2 : of.W3);
            const int ob = layer == 0 ? of.b1 : (layer == 1 ? of.b2 : of.b3);
            dst = ii < K ? ow + oo * K + ii : ob + oo;
        }
        G[dst] = acc[k];
    }
}

// Adam (Kingma & Ba) with the step count kept on the device: step s = *count + 1.
__global__ void k_mlp_adam(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                           float *__restrict__ V, int n, float lr, float beta1, float beta2, float eps,
                           const unsigned *__restrict__ count) {
    const unsigned s = *count + 1u;
    const float bc1 = (float)(1.0 - pow((double)beta1, (double)s));
    const float bc2 = (float)(1.0 - pow((double)beta2, (double)s));
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const float g = G[j];
        const float m = fmaf(beta1, M[j], (1.f - beta1) * g);
        const float v = fmaf(beta2, V[j], (1.f - beta2) * g * g);
        M[j] = m;
        V[j] = v;
        const float mhat = m / bc1, vhat = v / bc2;
        P[j] -= lr * mhat / (sqrtf(vhat) + eps);
    }
}

__global__ void k_mlp_count(unsigned *count) { *count += 1u; }

// Glorot-uniform weights, zero biases: weight j takes u_j from the
// SplitMix64 stream of the seed (output j + 1) as a * (2 u_j - 1), a =
// sqrt(6 / (fan_in + fan_out)).
__device__ inline uint64_t splitmix_at(uint64_t seed, uint64_t k) {
    uint64_t zz = seed + k * 0x9E3779B97F4A7C15ull;
    zz = (zz ^ (zz >> 30)) * 0xBF58476D1CE4E5B9ull;
    zz = (zz ^ (zz >> 27)) * 0x94D049BB133111EBull;
    return zz ^ (zz >> 31);
}

__global__ void k_mlp_init(float *P, int n_in, uint64_t seed) {
    const Offsets of = offsets(n_in);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < of.total; j += gridDim.x * blockDim.x) {
        float a = 0.f;
        if (j < of.b1)
            a = sqrtf(6.f / (float)(n_in + W));
        else if ((j >= of.W2 && j < of.b2) || (j >= of.W3 && j < of.b3))
            a = sqrtf(6.f / (float)(W + W));
        else if (j >= of.wo && j < of.bo)
            a = sqrtf(6.f / (float)(W + 1));
        const double u = (double)(splitmix_at(seed, (uint64_t)j + 1) >> 11) * 0x1.0p-53;
        P[j] = a == 0.f ? 0.f : (float)((double)a * (2.0 * u - 1.0));
    }
}

}  // namespace

int mlp_num_params(int n_in) { return offsets(n_in).total; }
int mlp_wgrad_tiles() { return 49; }

size_t mlp_forward_smem() { return sizeof(float) * ((size_t)W * WS_STRIDE + 2 * ROWS * W); }

int mlp_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mlp_forward_smem());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_forward_smem());
    return (int)e;
}

int mlp_launch_init(float *P, int n_in, uint64_t seed, void *stream) {
    k_mlp_init<<<64, 256, 0, (cudaStream_t)stream>>>(P, n_in, seed);
    return (int)cudaGetLastError();
}

int mlp_launch_standardize(const float *x, const float *y, int rows, int n_in, const MlpNorm &nm, float *xs,
                           float *ys, void *stream) {
    const int total = rows * n_in;
    int blocks = (total + 255) / 256;
    blocks = blocks < 1 ? 1 : (blocks > 1024 ? 1024 : blocks);
    k_mlp_standardize<<<blocks, 256, 0, (cudaStream_t)stream>>>(x, y, rows, n_in, nm, xs, ys);
    return (int)cudaGetLastError();
}

int mlp_launch_forward(const float *P, const float *xs, const int *idx, int rows, int n_in, float *acts, float *out,
                       int denorm, float y_mu, float y_sigma, void *stream) {
    if (rows <= 0) return 0;
    k_mlp_forward<<<(rows + ROWS - 1) / ROWS, THREADS, mlp_forward_smem(), (cudaStream_t)stream>>>(
        P, xs, idx, rows, n_in, acts, out, denorm, y_mu, y_sigma);
    return (int)cudaGetLastError();
}

int mlp_launch_backward(const float *P, const float *ts, const int *idx, int rows, int n_in, float inv_B,
                        const float *acts, const float *out, float *deltas, float *loss_part, void *stream) {
    if (rows <= 0) return 0;
    k_mlp_backward<<<(rows + ROWS - 1) / ROWS, THREADS, mlp_forward_smem(), (cudaStream_t)stream>>>(
        P, ts, idx, rows, n_in, inv_B, acts, out, deltas, loss_part);
    return (int)cudaGetLastError();
}

int mlp_launch_wgrad(const float *xs, const int *idx, int rows, int n_in, const float *acts, const float *deltas,
                     float *G, void *stream) {
    k_mlp_wgrad<<<mlp_wgrad_tiles(), THREADS, 0, (cudaStream_t)stream>>>(xs, idx, rows, n_in, acts, deltas, G);
    return (int)cudaGetLastError();
}

int mlp_launch_adam(float *P, const float *G, float *M, float *V, int n, float lr, float beta1, float beta2,
                    float eps, unsigned *count, void *stream) {
    k_mlp_adam<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(P, G, M, V, n, lr, beta1, beta2, eps, count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    k_mlp_count<<<1, 1, 0, (cudaStream_t)stream>>>(count);
    return (int)cudaGetLastError();
}

}  // namespace ps
