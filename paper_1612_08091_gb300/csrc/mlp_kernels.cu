// mlp_kernels.cu -- the cost model behind the learned fusion planner:
// a 3-layer perceptron  x (16) -> relu(W1 x + b1) (H) -> relu(W2 h1 + b2) (H)
// -> w3 . h2 + b3 (1),  trained on the GPU with these kernels.
//
// Not a method of the paper.  Its inputs are the features of one unit of
// planned device work (a fused block or a plain gate launch; see planner.cpp)
// and its output is the predicted log of that launch's duration in ms.  The
// training targets are durations the simulator measured itself with CUDA
// events (sim_get_item_times).
//
// Everything is FP32 and deterministic: weight gradients are sums over the
// batch in sample order, one thread per weight, no atomics.  The kernels
// are small dense loops on the CUDA cores; the matrices are far too small
// for the tensor cores to matter.
//
// Parameter vector layout (P = H*16 + H + H*H + H + H + 1 floats):
//   W1 [H][16], b1 [H], W2 [H][H], b2 [H], w3 [H], b3.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/qsim.h"

namespace {

constexpr int kIn = 16;

struct Dims {
    int H;
    size_t oW1, ob1, oW2, ob2, ow3, ob3, P;
};

Dims dims(int H) {
    Dims d;
    d.H = H;
    d.oW1 = 0;
    d.ob1 = d.oW1 + (size_t)H * kIn;
    d.oW2 = d.ob1 + H;
    d.ob2 = d.oW2 + (size_t)H * H;
    d.ow3 = d.ob2 + H;
    d.ob3 = d.ow3 + H;
    d.P = d.ob3 + 1;
    return d;
}

// Y[b][j] = act( sum_i X[b][i] W[j][i] + bias[j] ),  one thread per (b, j)
__global__ void k_linear_fwd(const float *__restrict__ X, const float *__restrict__ W, const float *__restrict__ bias,
                             float *__restrict__ Y, int B, int in, int out, int relu) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * out) return;
    const int b = idx / out, j = idx % out;
    float acc = bias[j];
    for (int i = 0; i < in; ++i) acc = fmaf(X[(size_t)b * in + i], W[(size_t)j * in + i], acc);
    Y[idx] = relu ? fmaxf(acc, 0.f) : acc;
}

// dY[b] = 2 (Y[b] - T[b]) / B  and the per-sample squared error
__global__ void k_mse_grad(const float *__restrict__ Y, const float *__restrict__ T, float *__restrict__ dY,
                           float *__restrict__ sq, int B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float d = Y[b] - T[b];
    dY[b] = 2.f * d / (float)B;
    sq[b] = d * d;
}

// dX[b][i] = (sum_j dY[b][j] W[j][i]) * (Xact[b][i] > 0 if mask)
__global__ void k_linear_bwd_data(const float *__restrict__ dY, const float *__restrict__ W,
                                  const float *__restrict__ Xact, float *__restrict__ dX, int B, int in, int out,
                                  int mask) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * in) return;
    const int b = idx / in, i = idx % in;
    float acc = 0.f;
    for (int j = 0; j < out; ++j) acc = fmaf(dY[(size_t)b * out + j], W[(size_t)j * in + i], acc);
    if (mask && !(Xact[idx] > 0.f)) acc = 0.f;
    dX[idx] = acc;
}

// dW[j][i] = sum_b dY[b][j] X[b][i];  db[j] = sum_b dY[b][j]  (batch order)
__global__ void k_linear_bwd_weight(const float *__restrict__ dY, const float *__restrict__ X, float *__restrict__ dW,
                                    float *__restrict__ db, int B, int in, int out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < out * in) {
        const int j = idx / in, i = idx % in;
        float acc = 0.f;
        for (int b = 0; b < B; ++b) acc = fmaf(dY[(size_t)b * out + j], X[(size_t)b * in + i], acc);
        dW[idx] = acc;
    } else if (idx < out * in + out) {
        const int j = idx - out * in;
        float acc = 0.f;
        for (int b = 0; b < B; ++b) acc += dY[(size_t)b * out + j];
        db[j] = acc;
    }
}

// Adam (bias-corrected)
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

unsigned blocks(size_t work, int t = 256) { return (unsigned)((work + t - 1) / t); }

}  // namespace

struct qsim_mlp {
    Dims d;
    int cap = 0;  // batch capacity of the activation buffers
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    float *X = nullptr, *T = nullptr, *H1 = nullptr, *H2 = nullptr, *Y = nullptr;
    float *dY = nullptr, *dH2 = nullptr, *dH1 = nullptr, *sq = nullptr;
    long long step = 0;
    cudaStream_t stream = nullptr;
    std::string err;
};

namespace {

int mlp_err(qsim_mlp *m, int code, const char *msg) {
    if (m) m->err = msg;
    return code;
}

int ensure_capacity(qsim_mlp *m, int B) {
    if (B <= m->cap) return QSIM_OK;
    const int H = m->d.H;
    float **bufs[] = {&m->X, &m->T, &m->H1, &m->H2, &m->Y, &m->dY, &m->dH2, &m->dH1, &m->sq};
    const size_t sizes[] = {(size_t)B * kIn, (size_t)B, (size_t)B * H, (size_t)B * H, (size_t)B,
                            (size_t)B, (size_t)B * H, (size_t)B * H, (size_t)B};
    for (int i = 0; i < 9; ++i) {
        if (*bufs[i]) cudaFree(*bufs[i]);
        *bufs[i] = nullptr;
        if (cudaMalloc((void **)bufs[i], sizeof(float) * sizes[i]) != cudaSuccess) {
            cudaGetLastError();
            m->cap = 0;
            return mlp_err(m, QSIM_ENOMEM, "activation buffers");
        }
    }
    m->cap = B;
    return QSIM_OK;
}

// forward on m->X (B samples) into H1, H2, Y
void forward(qsim_mlp *m, int B) {
    const Dims &d = m->d;
    const int H = d.H;
    k_linear_fwd<<<blocks((size_t)B * H), 256, 0, m->stream>>>(m->X, m->params + d.oW1, m->params + d.ob1, m->H1, B,
                                                                 kIn, H, 1);
    k_linear_fwd<<<blocks((size_t)B * H), 256, 0, m->stream>>>(m->H1, m->params + d.oW2, m->params + d.ob2, m->H2, B,
                                                                 H, H, 1);
    k_linear_fwd<<<blocks((size_t)B), 256, 0, m->stream>>>(m->H2, m->params + d.ow3, m->params + d.ob3, m->Y, B, H, 1,
                                                             0);
}

// gradients of the mean squared error into m->grads (after forward)
void backward(qsim_mlp *m, int B) {
    const Dims &d = m->d;
    const int H = d.H;
    k_mse_grad<<<blocks(B), 256, 0, m->stream>>>(m->Y, m->T, m->dY, m->sq, B);
    k_linear_bwd_weight<<<blocks((size_t)H + 1), 256, 0, m->stream>>>(m->dY, m->H2, m->grads + d.ow3,
                                                                        m->grads + d.ob3, B, H, 1);
    k_linear_bwd_data<<<blocks((size_t)B * H), 256, 0, m->stream>>>(m->dY, m->params + d.ow3, m->H2, m->dH2, B, H, 1,
                                                                      1);
    k_linear_bwd_weight<<<blocks((size_t)H * H + H), 256, 0, m->stream>>>(m->dH2, m->H1, m->grads + d.oW2,
                                                                            m->grads + d.ob2, B, H, H);
    k_linear_bwd_data<<<blocks((size_t)B * H), 256, 0, m->stream>>>(m->dH2, m->params + d.oW2, m->H1, m->dH1, B, H,
                                                                      H, 1);
    k_linear_bwd_weight<<<blocks((size_t)H * kIn + H), 256, 0, m->stream>>>(m->dH1, m->X, m->grads + d.oW1,
                                                                              m->grads + d.ob1, B, kIn, H);
}

// splitmix64 -> uniform in [-1, 1)
double mix_uniform(unsigned long long &state) {
    unsigned long long z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

}  // namespace

extern "C" {

int sim_mlp_param_count(int hidden) { return hidden >= 1 && hidden <= 1024 ? (int)dims(hidden).P : -1; }

int sim_mlp_create(int hidden, unsigned long long seed, void *stream, qsim_mlp **out) {
    if (!out || hidden < 1 || hidden > 1024) return QSIM_EINVAL;
    *out = nullptr;
    qsim_mlp *m = new (std::nothrow) qsim_mlp();
    if (!m) return QSIM_ENOMEM;
    m->d = dims(hidden);
    m->stream = (cudaStream_t)stream;
    const size_t P = m->d.P;
    float **bufs[] = {&m->params, &m->grads, &m->m, &m->v};
    for (float **b : bufs) {
        if (cudaMalloc((void **)b, sizeof(float) * P) != cudaSuccess) {
            cudaGetLastError();
            sim_mlp_destroy(m);
            return QSIM_ENOMEM;
        }
    }
    // He-uniform weights, zero biases, from a seeded splitmix64 stream
    std::vector<float> p(P, 0.f);
    unsigned long long st = seed;
    const int H = hidden;
    const double a1 = std::sqrt(6.0 / kIn), a2 = std::sqrt(6.0 / H);
    for (size_t i = 0; i < (size_t)H * kIn; ++i) p[m->d.oW1 + i] = (float)(a1 * mix_uniform(st));
    for (size_t i = 0; i < (size_t)H * H; ++i) p[m->d.oW2 + i] = (float)(a2 * mix_uniform(st));
    for (int i = 0; i < H; ++i) p[m->d.ow3 + i] = (float)(a2 * mix_uniform(st));
    cudaMemcpyAsync(m->params, p.data(), sizeof(float) * P, cudaMemcpyHostToDevice, m->stream);
    cudaMemsetAsync(m->m, 0, sizeof(float) * P, m->stream);
    cudaMemsetAsync(m->v, 0, sizeof(float) * P, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        sim_mlp_destroy(m);
        return QSIM_ECUDA;
    }
    *out = m;
    return QSIM_OK;
}

int sim_mlp_destroy(qsim_mlp *m) {
    if (!m) return QSIM_OK;
    if (m->stream) cudaStreamSynchronize(m->stream);
    float *bufs[] = {m->params, m->grads, m->m, m->v, m->X, m->T, m->H1, m->H2, m->Y, m->dY, m->dH2, m->dH1, m->sq};
    for (float *b : bufs)
        if (b) cudaFree(b);
    delete m;
    return QSIM_OK;
}

int sim_mlp_get_params(qsim_mlp *m, float *out, int count) {
    if (!m || !out || count != (int)m->d.P) return QSIM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(out, m->params, sizeof(float) * count, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? QSIM_OK : QSIM_ECUDA;
}

int sim_mlp_set_params(qsim_mlp *m, const float *in, int count) {
    if (!m || !in || count != (int)m->d.P) return QSIM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(m->params, in, sizeof(float) * count, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    return e == cudaSuccess ? QSIM_OK : QSIM_ECUDA;
}

int sim_mlp_forward(qsim_mlp *m, const float *X, int n, float *Y) {
    if (!m || n < 1 || !X || !Y) return QSIM_EINVAL;
    int rc = ensure_capacity(m, n);
    if (rc) return rc;
    cudaMemcpyAsync(m->X, X, sizeof(float) * n * kIn, cudaMemcpyHostToDevice, m->stream);
    forward(m, n);
    cudaMemcpyAsync(Y, m->Y, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream);
    return cudaStreamSynchronize(m->stream) == cudaSuccess ? QSIM_OK : QSIM_ECUDA;
}

// Gradient of the mean squared error over the n samples (for checking).
int sim_mlp_gradient(qsim_mlp *m, const float *X, const float *T, int n, float *grads, float *loss) {
    if (!m || n < 1 || !X || !T || !grads) return QSIM_EINVAL;
    int rc = ensure_capacity(m, n);
    if (rc) return rc;
    cudaMemcpyAsync(m->X, X, sizeof(float) * n * kIn, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(m->T, T, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream);
    forward(m, n);
    backward(m, n);
    std::vector<float> sq(n);
    cudaMemcpyAsync(grads, m->grads, sizeof(float) * m->d.P, cudaMemcpyDeviceToHost, m->stream);
    cudaMemcpyAsync(sq.data(), m->sq, sizeof(float) * n, cudaMemcpyDeviceToHost, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return QSIM_ECUDA;
    if (loss) {
        double s = 0.0;
        for (float v : sq) s += v;
        *loss = (float)(s / n);
    }
    return QSIM_OK;
}

// Adam on the mean squared error: `epochs` passes over the n samples in
// minibatches of `batch` (in order, last one partial).  *loss receives the
// mean squared error of the final epoch.
int sim_mlp_train(qsim_mlp *m, const float *X, const float *T, int n, int epochs, int batch, float lr, float *loss) {
    if (!m || n < 1 || !X || !T || epochs < 1 || batch < 1 || !(lr > 0.f)) return QSIM_EINVAL;
    if (batch > n) batch = n;
    int rc = ensure_capacity(m, n);
    if (rc) return rc;
    // all samples resident on the device; minibatches are views
    float *Xall = nullptr, *Tall = nullptr;
    if (cudaMalloc((void **)&Xall, sizeof(float) * n * kIn) != cudaSuccess ||
        cudaMalloc((void **)&Tall, sizeof(float) * n) != cudaSuccess) {
        cudaGetLastError();
        if (Xall) cudaFree(Xall);
        return mlp_err(m, QSIM_ENOMEM, "training set");
    }
    cudaMemcpyAsync(Xall, X, sizeof(float) * n * kIn, cudaMemcpyHostToDevice, m->stream);
    cudaMemcpyAsync(Tall, T, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream);
    float *keepX = m->X, *keepT = m->T;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double last = 0.0;
    std::vector<float> sq;
    for (int ep = 0; ep < epochs; ++ep) {
        double ep_sum = 0.0;
        for (int s0 = 0; s0 < n; s0 += batch) {
            const int B = std::min(batch, n - s0);
            m->X = Xall + (size_t)s0 * kIn;
            m->T = Tall + s0;
            forward(m, B);
            backward(m, B);
            ++m->step;
            const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
            k_adam<<<blocks(m->d.P), 256, 0, m->stream>>>(m->params, m->grads, m->m, m->v, (int)m->d.P, lr, b1, b2,
                                                          eps, c1, c2);
            if (ep == epochs - 1) {
                sq.resize(B);
                cudaMemcpyAsync(sq.data(), m->sq, sizeof(float) * B, cudaMemcpyDeviceToHost, m->stream);
                cudaStreamSynchronize(m->stream);
                for (float v : sq) ep_sum += v;
            }
        }
        if (ep == epochs - 1) last = ep_sum / n;
    }
    m->X = keepX;
    m->T = keepT;
    cudaError_t e = cudaStreamSynchronize(m->stream);
    cudaFree(Xall);
    cudaFree(Tall);
    if (e != cudaSuccess) return mlp_err(m, QSIM_ECUDA, cudaGetErrorString(e));
    if (loss) *loss = (float)last;
    return QSIM_OK;
}

}  // extern "C"
