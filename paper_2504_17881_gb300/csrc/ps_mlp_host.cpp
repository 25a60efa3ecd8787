// The step-count predictor object (include/ps.h): parameters and Adam state
// on the device, training epochs replayed from a CUDA graph, inference, and
// the choice of the Trotter step count r from the predicted log error.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <sstream>
#include <vector>

#include "ps_internal.h"

namespace ps {
namespace {

int mfail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

int cuda_mfail(cudaError_t e, const char *what) {
    std::ostringstream os;
    os << what << ": " << cudaGetErrorName(e) << " (" << cudaGetErrorString(e) << ")";
    return mfail(e == cudaErrorMemoryAllocation ? PS_ERR_OOM : PS_ERR_CUDA, os.str());
}

uint64_t splitmix_next(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace
}  // namespace ps

using namespace ps;

struct ps_mlp {
    int n_in = 0;
    int nparams = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    MlpNorm norm{};
    float y_sigma = 1.f;
    // device: parameters, gradients, Adam moments, Adam step count
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    unsigned *count = nullptr;
    // workspace for up to cap rows
    size_t cap = 0;
    float *xs = nullptr, *ts = nullptr, *acts = nullptr, *deltas = nullptr, *out = nullptr, *loss_part = nullptr;
    int *idx = nullptr;
    float *h_loss = nullptr;  // pinned, cap_loss floats
    int *h_idx = nullptr;     // pinned, cap ints
    size_t cap_loss = 0;
};

namespace {

void free_ws(ps_mlp *m) {
    for (float *p : {m->xs, m->ts, m->acts, m->deltas, m->out, m->loss_part})
        if (p) cudaFree(p);
    if (m->idx) cudaFree(m->idx);
    if (m->h_idx) cudaFreeHost(m->h_idx);
    m->xs = m->ts = m->acts = m->deltas = m->out = m->loss_part = nullptr;
    m->idx = nullptr;
    m->h_idx = nullptr;
    m->cap = 0;
}

// Room for `rows` rows (dataset copies, activations, deltas, outputs).
int ensure(ps_mlp *m, size_t rows) {
    if (rows <= m->cap) return PS_OK;
    cudaStreamSynchronize(m->stream);
    free_ws(m);
    const size_t W = kMlpWidth;
    cudaError_t e = cudaMalloc((void **)&m->xs, sizeof(float) * rows * m->n_in);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->ts, sizeof(float) * rows);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->acts, sizeof(float) * 3 * rows * W);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->deltas, sizeof(float) * (3 * rows * W + rows));
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->out, sizeof(float) * rows);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->loss_part, sizeof(float) * (rows / 32 + 2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->idx, sizeof(int) * rows);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&m->h_idx, sizeof(int) * rows);
    if (e != cudaSuccess) {
        free_ws(m);
        return cuda_mfail(e, "MLP workspace allocation");
    }
    m->cap = rows;
    return PS_OK;
}

int ensure_loss(ps_mlp *m, size_t n) {
    if (n <= m->cap_loss) return PS_OK;
    if (m->h_loss) cudaFreeHost(m->h_loss);
    m->h_loss = nullptr;
    m->cap_loss = 0;
    cudaError_t e = cudaMallocHost((void **)&m->h_loss, sizeof(float) * n);
    if (e != cudaSuccess) return cuda_mfail(e, "MLP loss buffer");
    m->cap_loss = n;
    return PS_OK;
}

int check_rows(size_t rows) {
    if (rows == 0) return mfail(PS_ERR_ARG, "rows must be >= 1");
    if (rows > (size_t)1 << 26) return mfail(PS_ERR_ARG, "at most 2^26 rows");
    return PS_OK;
}

struct Guard {
    int prev = -1;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Forward, backward and weight gradients of `rows` rows (indices idx into
// the standardised dataset, or the rows in order) into m->G; per-CTA sums of
// squared errors into loss_part.
int grad_pass(ps_mlp *m, const int *idx, int rows, float *loss_part, cudaStream_t s) {
    int e = mlp_launch_forward(m->P, m->xs, idx, rows, m->n_in, m->acts, m->out, 0, 0.f, 1.f, s);
    if (e == 0)
        e = mlp_launch_backward(m->P, m->ts, idx, rows, m->n_in, 1.f / (float)rows, m->acts, m->out, m->deltas,
                                loss_part, s);
    if (e == 0) e = mlp_launch_wgrad(m->xs, idx, rows, m->n_in, m->acts, m->deltas, m->G, s);
    return e;
}

}  // namespace

extern "C" {

int ps_mlp_create(int n_in, uint64_t seed, void *stream, ps_mlp **out) {
    if (!out) return mfail(PS_ERR_ARG, "null output pointer");
    *out = nullptr;
    if (n_in < 1 || n_in > kMlpMaxIn) return mfail(PS_ERR_ARG, "n_in must be in [1, 16]");
    ps_mlp *m = new (std::nothrow) ps_mlp();
    if (!m) return mfail(PS_ERR_OOM, "host allocation failed");
    m->n_in = n_in;
    m->nparams = mlp_num_params(n_in);
    m->stream = (cudaStream_t)stream;
    for (int i = 0; i < kMlpMaxIn; ++i) {
        m->norm.mu[i] = 0.f;
        m->norm.inv_sigma[i] = 1.f;
    }
    m->norm.y_mu = 0.f;
    m->norm.y_inv_sigma = 1.f;
    cudaError_t e = cudaGetDevice(&m->device);
    const size_t bytes = sizeof(float) * (size_t)m->nparams;
    if (e == cudaSuccess) e = (cudaError_t)mlp_prepare();
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->P, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->G, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->M, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->V, bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m->count, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(m->G, 0, bytes, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->M, 0, bytes, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->V, 0, bytes, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->count, 0, sizeof(unsigned), m->stream);
    if (e == cudaSuccess) e = (cudaError_t)mlp_launch_init(m->P, n_in, seed, m->stream);
    if (e != cudaSuccess) {
        const int rc = cuda_mfail(e, "ps_mlp_create");
        ps_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return PS_OK;
}

void ps_mlp_destroy(ps_mlp *m) {
    if (!m) return;
    Guard g(m->device);
    cudaStreamSynchronize(m->stream);
    free_ws(m);
    if (m->h_loss) cudaFreeHost(m->h_loss);
    for (float *p : {m->P, m->G, m->M, m->V})
        if (p) cudaFree(p);
    if (m->count) cudaFree(m->count);
    delete m;
}

size_t ps_mlp_num_params(const ps_mlp *m) { return m ? (size_t)m->nparams : 0; }

static int copy_params(ps_mlp *m, float *dst_host, const float *src_dev) {
    Guard g(m->device);
    cudaError_t e = cudaMemcpyAsync(dst_host, src_dev, sizeof(float) * m->nparams, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? PS_OK : cuda_mfail(e, "MLP parameter readback");
}

int ps_mlp_get_params(ps_mlp *m, float *host) {
    if (!m || !host) return mfail(PS_ERR_ARG, "null argument");
    return copy_params(m, host, m->P);
}

int ps_mlp_get_grads(ps_mlp *m, float *host) {
    if (!m || !host) return mfail(PS_ERR_ARG, "null argument");
    return copy_params(m, host, m->G);
}

int ps_mlp_set_grads(ps_mlp *m, const float *host) {
    if (!m || !host) return mfail(PS_ERR_ARG, "null argument");
    Guard g(m->device);
    cudaError_t e = cudaMemcpyAsync(m->G, host, sizeof(float) * m->nparams, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e != cudaSuccess ? cuda_mfail(e, "ps_mlp_set_grads") : PS_OK;
}

int ps_mlp_set_params(ps_mlp *m, const float *host) {
    if (!m || !host) return mfail(PS_ERR_ARG, "null argument");
    Guard g(m->device);
    cudaError_t e = cudaMemcpyAsync(m->P, host, sizeof(float) * m->nparams, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? PS_OK : cuda_mfail(e, "MLP parameter upload");
}

int ps_mlp_set_normalization(ps_mlp *m, const float *mu, const float *sigma, float y_mu, float y_sigma) {
    if (!m || !mu || !sigma) return mfail(PS_ERR_ARG, "null argument");
    for (int i = 0; i < m->n_in; ++i)
        if (!(sigma[i] > 0.f) || !std::isfinite(mu[i])) return mfail(PS_ERR_ARG, "sigma must be positive");
    if (!(y_sigma > 0.f) || !std::isfinite(y_mu)) return mfail(PS_ERR_ARG, "y_sigma must be positive");
    for (int i = 0; i < m->n_in; ++i) {
        m->norm.mu[i] = mu[i];
        m->norm.inv_sigma[i] = 1.f / sigma[i];
    }
    m->norm.y_mu = y_mu;
    m->norm.y_inv_sigma = 1.f / y_sigma;
    m->y_sigma = y_sigma;
    return PS_OK;
}

int ps_mlp_get_normalization(const ps_mlp *m, float *mu, float *sigma, float *y_mu, float *y_sigma) {
    if (!m) return mfail(PS_ERR_ARG, "null argument");
    for (int i = 0; i < m->n_in; ++i) {
        if (mu) mu[i] = m->norm.mu[i];
        if (sigma) sigma[i] = 1.f / m->norm.inv_sigma[i];
    }
    if (y_mu) *y_mu = m->norm.y_mu;
    if (y_sigma) *y_sigma = m->y_sigma;
    return PS_OK;
}

int ps_mlp_fit_normalization(ps_mlp *m, const float *x, const float *y, size_t rows) {
    if (!m || !x || !y) return mfail(PS_ERR_ARG, "null argument");
    if (int rc = check_rows(rows)) return rc;
    // mean and standard deviation per column, FP64, rows in order
    std::vector<double> mu(m->n_in, 0.0), var(m->n_in, 0.0);
    double ym = 0.0, yv = 0.0;
    for (size_t r = 0; r < rows; ++r) {
        for (int i = 0; i < m->n_in; ++i) mu[i] += x[r * m->n_in + i];
        ym += y[r];
    }
    for (int i = 0; i < m->n_in; ++i) mu[i] /= (double)rows;
    ym /= (double)rows;
    for (size_t r = 0; r < rows; ++r) {
        for (int i = 0; i < m->n_in; ++i) {
            const double d = x[r * m->n_in + i] - mu[i];
            var[i] += d * d;
        }
        yv += (y[r] - ym) * (y[r] - ym);
    }
    std::vector<float> fm(m->n_in), fs(m->n_in);
    for (int i = 0; i < m->n_in; ++i) {
        fm[i] = (float)mu[i];
        const double sd = std::sqrt(var[i] / (double)rows);
        fs[i] = sd > 1e-12 ? (float)sd : 1.f;  // a constant column stays unscaled
    }
    const double ysd = std::sqrt(yv / (double)rows);
    return ps_mlp_set_normalization(m, fm.data(), fs.data(), (float)ym, ysd > 1e-12 ? (float)ysd : 1.f);
}

int ps_mlp_loss_grad(ps_mlp *m, const float *x_dev, const float *y_dev, size_t rows, double *loss_out) {
    if (!m || !x_dev || !y_dev) return mfail(PS_ERR_ARG, "null argument");
    if (int rc = check_rows(rows)) return rc;
    Guard g(m->device);
    if (int rc = ensure(m, rows)) return rc;
    const size_t nb = (rows + 31) / 32;
    if (int rc = ensure_loss(m, nb)) return rc;
    int e = mlp_launch_standardize(x_dev, y_dev, (int)rows, m->n_in, m->norm, m->xs, m->ts, m->stream);
    if (e == 0) e = grad_pass(m, nullptr, (int)rows, m->loss_part, m->stream);
    if (e) return cuda_mfail((cudaError_t)e, "MLP gradient kernels");
    cudaError_t ce = cudaMemcpyAsync(m->h_loss, m->loss_part, sizeof(float) * nb, cudaMemcpyDeviceToHost, m->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(m->stream);
    if (ce != cudaSuccess) return cuda_mfail(ce, "MLP loss readback");
    double s = 0.0;
    for (size_t b = 0; b < nb; ++b) s += m->h_loss[b];
    if (loss_out) *loss_out = s / (double)rows;
    return PS_OK;
}

int ps_mlp_adam_step(ps_mlp *m, float lr, float beta1, float beta2, float eps) {
    if (!m) return mfail(PS_ERR_ARG, "null argument");
    if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return mfail(PS_ERR_ARG, "invalid Adam hyper-parameters");
    Guard g(m->device);
    const int e = mlp_launch_adam(m->P, m->G, m->M, m->V, m->nparams, lr, beta1, beta2, eps, m->count, m->stream);
    return e ? cuda_mfail((cudaError_t)e, "Adam kernel") : PS_OK;
}

int ps_mlp_train(ps_mlp *m, const float *x_dev, const float *y_dev, size_t rows, const ps_mlp_train_config *cfg,
                 float *loss_per_epoch) {
    if (!m || !x_dev || !y_dev) return mfail(PS_ERR_ARG, "null argument");
    if (int rc = check_rows(rows)) return rc;
    const int epochs = (cfg && cfg->epochs) ? cfg->epochs : 200;
    int batch = (cfg && cfg->batch) ? cfg->batch : 256;
    const float lr = (cfg && cfg->lr > 0.f) ? cfg->lr : 1e-3f;
    const float b1 = (cfg && cfg->beta1 > 0.f) ? cfg->beta1 : 0.9f;
    const float b2 = (cfg && cfg->beta2 > 0.f) ? cfg->beta2 : 0.999f;
    const float eps = (cfg && cfg->eps > 0.f) ? cfg->eps : 1e-8f;
    const uint64_t seed = cfg ? cfg->seed : 0;
    if (epochs < 1 || epochs > 1000000) return mfail(PS_ERR_ARG, "epochs must be in [1, 1e6]");
    if (batch < 1) return mfail(PS_ERR_ARG, "batch must be >= 1");
    if (b1 >= 1.f || b2 >= 1.f) return mfail(PS_ERR_ARG, "invalid Adam hyper-parameters");
    if ((size_t)batch > rows) batch = (int)rows;
    const int steps = (int)(rows / (size_t)batch);  // the last partial batch of an epoch is dropped
    const int nb = (batch + 31) / 32;
    Guard g(m->device);
    if (int rc = ensure(m, rows)) return rc;
    if (int rc = ensure_loss(m, (size_t)steps * nb)) return rc;
    // the loss partials of every step of an epoch
    float *parts = nullptr;
    cudaError_t ce = cudaMalloc((void **)&parts, sizeof(float) * (size_t)steps * nb);
    if (ce != cudaSuccess) return cuda_mfail(ce, "MLP training buffers");
    int e = mlp_launch_standardize(x_dev, y_dev, (int)rows, m->n_in, m->norm, m->xs, m->ts, m->stream);
    if (e) {
        cudaFree(parts);
        return cuda_mfail((cudaError_t)e, "standardisation kernel");
    }
    // one epoch = `steps` x (forward, backward, weight gradients, Adam) over
    // consecutive slices of the permutation in m->idx, captured once
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int rc = PS_OK;
    ce = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        for (int s = 0; s < steps && e == 0; ++s) {
            e = grad_pass(m, m->idx + (size_t)s * batch, batch, parts + (size_t)s * nb, cap);
            if (e == 0) e = mlp_launch_adam(m->P, m->G, m->M, m->V, m->nparams, lr, b1, b2, eps, m->count, cap);
        }
        const cudaError_t ee = cudaStreamEndCapture(cap, &graph);
        if (e == 0 && ee != cudaSuccess) e = (int)ee;
        if (e == 0) e = (int)cudaGraphInstantiate(&exec, graph, 0);
    } else {
        e = (int)ce;
    }
    if (e) rc = cuda_mfail((cudaError_t)e, "MLP epoch graph");
    std::vector<int> perm(rows);
    for (int ep = 0; ep < epochs && rc == PS_OK; ++ep) {
        // Fisher-Yates shuffle from SplitMix64(seed, epoch)
        uint64_t st = seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(ep + 1));
        for (size_t i = 0; i < rows; ++i) perm[i] = (int)i;
        for (size_t i = rows - 1; i > 0; --i) {
            const size_t j = (size_t)(splitmix_next(st) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        cudaStreamSynchronize(m->stream);
        std::memcpy(m->h_idx, perm.data(), sizeof(int) * rows);
        ce = cudaMemcpyAsync(m->idx, m->h_idx, sizeof(int) * rows, cudaMemcpyHostToDevice, m->stream);
        if (ce == cudaSuccess) ce = cudaGraphLaunch(exec, m->stream);
        if (ce == cudaSuccess && loss_per_epoch)
            ce = cudaMemcpyAsync(m->h_loss, parts, sizeof(float) * (size_t)steps * nb, cudaMemcpyDeviceToHost,
                                 m->stream);
        if (ce == cudaSuccess && loss_per_epoch) ce = cudaStreamSynchronize(m->stream);
        if (ce != cudaSuccess) {
            rc = cuda_mfail(ce, "MLP training epoch");
            break;
        }
        if (loss_per_epoch) {
            double sum = 0.0;
            for (size_t k = 0; k < (size_t)steps * nb; ++k) sum += m->h_loss[k];
            loss_per_epoch[ep] = (float)(sum / ((double)steps * batch));
        }
    }
    cudaStreamSynchronize(m->stream);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    cudaFree(parts);
    return rc;
}

int ps_mlp_predict(ps_mlp *m, const float *x_dev, size_t rows, float *y_dev) {
    if (!m || !x_dev || !y_dev) return mfail(PS_ERR_ARG, "null argument");
    if (int rc = check_rows(rows)) return rc;
    Guard g(m->device);
    if (int rc = ensure(m, rows)) return rc;
    int e = mlp_launch_standardize(x_dev, nullptr, (int)rows, m->n_in, m->norm, m->xs, nullptr, m->stream);
    if (e == 0) e = mlp_launch_forward(m->P, m->xs, nullptr, (int)rows, m->n_in, nullptr, y_dev, 1, m->norm.y_mu,
                                       m->y_sigma, m->stream);
    return e ? cuda_mfail((cudaError_t)e, "MLP inference kernels") : PS_OK;
}

int ps_mlp_predict_ensemble(ps_mlp *const *nets, int count, const float *x_dev, size_t rows, float *y_host) {
    if (!nets || count < 1 || count > 64 || !x_dev || !y_host) return mfail(PS_ERR_ARG, "null argument or bad count");
    for (int k = 0; k < count; ++k) {
        if (!nets[k]) return mfail(PS_ERR_ARG, "null network");
        if (nets[k]->n_in != nets[0]->n_in || nets[k]->device != nets[0]->device)
            return mfail(PS_ERR_ARG, "members differ in inputs or device");
    }
    if (int rc = check_rows(rows)) return rc;
    Guard g(nets[0]->device);
    float *dy = nullptr;
    cudaError_t ce = cudaMalloc((void **)&dy, sizeof(float) * (size_t)count * rows);
    if (ce != cudaSuccess) return cuda_mfail(ce, "ensemble buffers");
    std::vector<float> all((size_t)count * rows);
    int rc = PS_OK;
    for (int k = 0; k < count && rc == PS_OK && ce == cudaSuccess; ++k) {
        rc = ps_mlp_predict(nets[k], x_dev, rows, dy + (size_t)k * rows);
        if (rc == PS_OK) ce = cudaStreamSynchronize(nets[k]->stream);
    }
    if (rc == PS_OK && ce == cudaSuccess)
        ce = cudaMemcpy(all.data(), dy, sizeof(float) * all.size(), cudaMemcpyDeviceToHost);
    cudaFree(dy);
    if (rc) return rc;
    if (ce != cudaSuccess) return cuda_mfail(ce, "ensemble transfer");
    // the mean of the members' log errors, in member order (as in ps_mlp_pick_r_ensemble)
    for (size_t i = 0; i < rows; ++i) {
        double s = 0.0;
        for (int k = 0; k < count; ++k) s += all[(size_t)k * rows + i];
        y_host[i] = (float)(s / count);
    }
    return PS_OK;
}

int ps_mlp_pick_r_ensemble(ps_mlp *const *nets, int count, ps_ham *ham, const uint64_t *idx, const double *amp,
                           size_t ndet, double t, double eps, double margin, uint32_t r_max, uint32_t *r_out,
                           float *pred_out) {
    if (!nets || count < 1 || count > 64 || !ham || !r_out) return mfail(PS_ERR_ARG, "null argument or bad count");
    for (int k = 0; k < count; ++k) {
        if (!nets[k]) return mfail(PS_ERR_ARG, "null network");
        if (nets[k]->n_in != kMlpFeatures) return mfail(PS_ERR_ARG, "the network must take the query features");
        if (nets[k]->device != nets[0]->device) return mfail(PS_ERR_ARG, "networks on different devices");
    }
    if (!(eps > 0.0)) return mfail(PS_ERR_ARG, "eps must be positive");
    if (r_max < 1 || r_max > (1u << 20)) return mfail(PS_ERR_ARG, "r_max must be in [1, 2^20]");
    *r_out = 0;
    std::vector<float> f((size_t)r_max * kMlpFeatures);
    for (uint32_t r = 1; r <= r_max; ++r)
        if (int rc = ham_query_features(ham, idx, amp, ndet, t, r, &f[(size_t)(r - 1) * kMlpFeatures])) return rc;
    ps_mlp *m0 = nets[0];
    Guard g(m0->device);
    float *d = nullptr;
    cudaError_t ce = cudaMalloc((void **)&d, sizeof(float) * ((size_t)r_max * kMlpFeatures + (size_t)count * r_max));
    if (ce != cudaSuccess) return cuda_mfail(ce, "pick_r buffers");
    float *dy = d + (size_t)r_max * kMlpFeatures;
    std::vector<float> all((size_t)count * r_max), pred(r_max, 0.f);
    int rc = PS_OK;
    ce = cudaMemcpyAsync(d, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice, m0->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(m0->stream);
    for (int k = 0; k < count && rc == PS_OK && ce == cudaSuccess; ++k) {
        rc = ps_mlp_predict(nets[k], d, r_max, dy + (size_t)k * r_max);
        if (rc == PS_OK) ce = cudaStreamSynchronize(nets[k]->stream);
    }
    if (rc == PS_OK && ce == cudaSuccess)
        ce = cudaMemcpy(all.data(), dy, sizeof(float) * all.size(), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (rc) return rc;
    if (ce != cudaSuccess) return cuda_mfail(ce, "pick_r transfer");
    // the ensemble's prediction: the mean of the members' log errors, in member order
    for (uint32_t r = 0; r < r_max; ++r) {
        double s = 0.0;
        for (int k = 0; k < count; ++k) s += all[(size_t)k * r_max + r];
        pred[r] = (float)(s / count);
    }
    if (pred_out) std::memcpy(pred_out, pred.data(), sizeof(float) * r_max);
    const double target = std::log(eps) - margin;
    for (uint32_t r = 1; r <= r_max; ++r)
        if ((double)pred[r - 1] <= target) {
            *r_out = r;
            return PS_OK;
        }
    std::ostringstream os;
    os << "no r <= " << r_max << " has a predicted log error below " << target;
    return mfail(PS_ERR_UNSUPPORTED, os.str());
}

int ps_mlp_pick_r(ps_mlp *m, ps_ham *ham, const uint64_t *idx, const double *amp, size_t ndet, double t, double eps,
                  double margin, uint32_t r_max, uint32_t *r_out, float *pred_out) {
    return ps_mlp_pick_r_ensemble(&m, 1, ham, idx, amp, ndet, t, eps, margin, r_max, r_out, pred_out);
}

}  // extern "C"
