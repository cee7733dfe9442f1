// Learned tuner: a small MLP (d_in -> h1 -> h2 -> sum(heads), ReLU, one
// softmax cross-entropy per head) with hand-written FP32 forward, backward and
// Adam kernels.  Every reduction over the batch is a fixed-order loop inside
// one thread, so training is deterministic.  The parameter blob layout is
// W1[h1][d_in], b1[h1], W2[h2][h1], b2[h2], W3[o][h2], b3[o].
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>

struct xb_mlp {
    int d_in = 0, h1 = 0, h2 = 0, nh = 0, o = 0;
    int heads[8] = {0};
    int64_t np = 0;
    float *d_param = nullptr, *d_grad = nullptr, *d_m = nullptr, *d_v = nullptr;
    float *d_norm = nullptr;  // mu[d_in], sd[d_in]
    int *d_heads = nullptr;
    float *d_act = nullptr;   // activation workspace
    size_t act_cap = 0;       // samples it holds
    float *d_loss = nullptr;  // per-sample loss
    float *d_xb = nullptr;    // minibatch features
    int *d_lb = nullptr;      // minibatch labels
    int *d_idx = nullptr;     // minibatch sample indices
    size_t mb_cap = 0;
    std::vector<float> h_mu, h_sd;
};

namespace {

struct Dims {
    int d_in, h1, h2, o, nh;
};

__device__ __forceinline__ const float *w1(const float *P, Dims d) { return P; }
__device__ __forceinline__ const float *b1(const float *P, Dims d) { return P + d.h1 * d.d_in; }
__device__ __forceinline__ const float *w2(const float *P, Dims d) { return b1(P, d) + d.h1; }
__device__ __forceinline__ const float *b2(const float *P, Dims d) { return w2(P, d) + d.h2 * d.h1; }
__device__ __forceinline__ const float *w3(const float *P, Dims d) { return b2(P, d) + d.h2; }
__device__ __forceinline__ const float *b3(const float *P, Dims d) { return w3(P, d) + d.o * d.h2; }

// Forward for one sample per thread; caches z1, z2 (pre-activations) and
// logits.  Inputs are standardised with (x - mu) / sd.
__global__ void k_fwd(int B, Dims d, const float *__restrict__ X, const float *__restrict__ norm,
                      const float *__restrict__ P, float *__restrict__ Z1, float *__restrict__ Z2,
                      float *__restrict__ L) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    float xn[16];
    for (int i = 0; i < d.d_in; i++) xn[i] = (X[(size_t)s * d.d_in + i] - norm[i]) / norm[d.d_in + i];
    float *z1 = Z1 + (size_t)s * d.h1, *z2 = Z2 + (size_t)s * d.h2, *lg = L + (size_t)s * d.o;
    const float *W1 = w1(P, d), *B1 = b1(P, d), *W2 = w2(P, d), *B2 = b2(P, d), *W3 = w3(P, d),
                *B3 = b3(P, d);
    for (int q = 0; q < d.h1; q++) {
        float a = B1[q];
        for (int i = 0; i < d.d_in; i++) a = fmaf(W1[q * d.d_in + i], xn[i], a);
        z1[q] = a;
    }
    for (int q = 0; q < d.h2; q++) {
        float a = B2[q];
        for (int i = 0; i < d.h1; i++) a = fmaf(W2[q * d.h1 + i], fmaxf(z1[i], 0.f), a);
        z2[q] = a;
    }
    for (int q = 0; q < d.o; q++) {
        float a = B3[q];
        for (int i = 0; i < d.h2; i++) a = fmaf(W3[q * d.h2 + i], fmaxf(z2[i], 0.f), a);
        lg[q] = a;
    }
}

// Softmax cross-entropy per head: dL/dlogit = (softmax - onehot) / B.
__global__ void k_xent(int B, Dims d, const int *__restrict__ heads, const float *__restrict__ L,
                       const int *__restrict__ lab, float *__restrict__ D3,
                       float *__restrict__ loss) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const float *lg = L + (size_t)s * d.o;
    float *g = D3 + (size_t)s * d.o;
    float ls = 0.f;
    int off = 0;
    for (int h = 0; h < d.nh; h++) {
        const int K = heads[h];
        float mx = lg[off];
        for (int c = 1; c < K; c++) mx = fmaxf(mx, lg[off + c]);
        float se = 0.f;
        for (int c = 0; c < K; c++) se += expf(lg[off + c] - mx);
        const int y = lab[(size_t)s * d.nh + h];
        if (y < 0) {  // no label for this head: no loss, no gradient
            for (int c = 0; c < K; c++) g[off + c] = 0.f;
            off += K;
            continue;
        }
        ls += -(lg[off + y] - mx - logf(se));
        for (int c = 0; c < K; c++)
            g[off + c] = (expf(lg[off + c] - mx) / se - (c == y ? 1.f : 0.f)) / (float)B;
        off += K;
    }
    loss[s] = ls / (float)B;
}

// gW[q][i] = sum_s D[s][q] * act(A[s][i]) (act = ReLU of the cached
// pre-activation, or the standardised input for the first layer);
// gb[q] = sum_s D[s][q].  One thread per (q, i) or per q for the bias.
__global__ void k_gw(int B, int out, int in, const float *__restrict__ D,
                     const float *__restrict__ A, int relu, const float *__restrict__ norm,
                     float *__restrict__ gW, float *__restrict__ gb) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < out * in) {
        const int q = t / in, i = t % in;
        float a = 0.f;
        for (int s = 0; s < B; s++) {
            float v = A[(size_t)s * in + i];
            v = relu ? fmaxf(v, 0.f) : (v - norm[i]) / norm[in + i];
            a = fmaf(D[(size_t)s * out + q], v, a);
        }
        gW[t] = a;
    } else if (t < out * in + out) {
        const int q = t - out * in;
        float a = 0.f;
        for (int s = 0; s < B; s++) a += D[(size_t)s * out + q];
        gb[q] = a;
    }
}

// Dprev[s][i] = (sum_q W[q][i] * D[s][q]) * [Z[s][i] > 0]
__global__ void k_back(int B, int out, int in, const float *__restrict__ W,
                       const float *__restrict__ D, const float *__restrict__ Z,
                       float *__restrict__ Dp) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * in) return;
    const int s = t / in, i = t % in;
    float a = 0.f;
    for (int q = 0; q < out; q++) a = fmaf(W[q * in + i], D[(size_t)s * out + q], a);
    Dp[t] = Z[t] > 0.f ? a : 0.f;
}

__global__ void k_adam(int64_t np, float *__restrict__ P, const float *__restrict__ G,
                       float *__restrict__ M, float *__restrict__ V, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M[i] + (1.f - b1) * g;
        const float v = b2 * V[i] + (1.f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

__global__ void k_gather_rows(int B, int w, const int *__restrict__ idx, const float *__restrict__ X,
                              float *__restrict__ Xb, const int *__restrict__ lab, int nh,
                              int *__restrict__ Lb) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    const int r = idx[s];
    for (int i = 0; i < w; i++) Xb[(size_t)s * w + i] = X[(size_t)r * w + i];
    for (int h = 0; h < nh; h++) Lb[(size_t)s * nh + h] = lab[(size_t)r * nh + h];
}

__global__ void k_argmax(int B, Dims d, const int *__restrict__ heads, const float *__restrict__ L,
                         int *__restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= B) return;
    int off = 0;
    for (int h = 0; h < d.nh; h++) {
        int best = 0;
        for (int c = 1; c < heads[h]; c++)
            if (L[(size_t)s * d.o + off + c] > L[(size_t)s * d.o + off + best]) best = c;
        out[(size_t)s * d.nh + h] = best;
        off += heads[h];
    }
}

__global__ void k_sum_loss(int B, const float *__restrict__ l, float *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float a = 0.f;
    for (int s = 0; s < B; s++) a += l[s];
    *out = a;
}

Dims dims_of(const xb_mlp *m) { return Dims{m->d_in, m->h1, m->h2, m->o, m->nh}; }

int ensure_act(xb_mlp *m, int B) {
    if ((size_t)B <= m->act_cap) return XB_OK;
    cudaFree(m->d_act);
    cudaFree(m->d_loss);
    m->d_act = nullptr;
    m->d_loss = nullptr;
    const size_t per = 2 * (size_t)m->h1 + 2 * (size_t)m->h2 + 2 * (size_t)m->o + 8;
    XB_CUDA(cudaMalloc(&m->d_act, per * B * sizeof(float)));
    XB_CUDA(cudaMalloc(&m->d_loss, ((size_t)B + 8) * sizeof(float)));
    m->act_cap = B;
    return XB_OK;
}

struct Act {
    float *z1, *z2, *lg, *d3, *d2, *d1;
};
Act act_of(xb_mlp *m) {
    Act a;
    const size_t C = m->act_cap;
    a.z1 = m->d_act;
    a.z2 = a.z1 + C * m->h1;
    a.lg = a.z2 + C * m->h2;
    a.d3 = a.lg + C * m->o;
    a.d2 = a.d3 + C * m->o;
    a.d1 = a.d2 + C * m->h2;
    return a;
}

int forward(xb_mlp *m, const float *X, int B, cudaStream_t s) {
    XB_TRY(ensure_act(m, B));
    Act a = act_of(m);
    k_fwd<<<(B + 127) / 128, 128, 0, s>>>(B, dims_of(m), X, m->d_norm, m->d_param, a.z1, a.z2, a.lg);
    XB_LAUNCHED("k_fwd");
    return XB_OK;
}

// loss and gradient of the batch into m->d_grad; loss sum into dev_loss
int loss_grad(xb_mlp *m, const float *X, const int *lab, int B, float *dev_loss, cudaStream_t s) {
    XB_TRY(forward(m, X, B, s));
    Act a = act_of(m);
    const Dims d = dims_of(m);
    k_xent<<<(B + 127) / 128, 128, 0, s>>>(B, d, m->d_heads, a.lg, lab, a.d3, m->d_loss);
    k_sum_loss<<<1, 32, 0, s>>>(B, m->d_loss, dev_loss);
    float *g = m->d_grad;
    float *gW1 = g, *gb1 = gW1 + m->h1 * m->d_in, *gW2 = gb1 + m->h1, *gb2 = gW2 + m->h2 * m->h1,
          *gW3 = gb2 + m->h2, *gb3 = gW3 + m->o * m->h2;
    const float *P = m->d_param;
    const float *W2 = P + m->h1 * m->d_in + m->h1, *W3 = W2 + m->h2 * m->h1 + m->h2;
    auto nb = [](int t) { return (t + 127) / 128; };
    k_gw<<<nb(m->o * m->h2 + m->o), 128, 0, s>>>(B, m->o, m->h2, a.d3, a.z2, 1, nullptr, gW3, gb3);
    k_back<<<nb(B * m->h2), 128, 0, s>>>(B, m->o, m->h2, W3, a.d3, a.z2, a.d2);
    k_gw<<<nb(m->h2 * m->h1 + m->h2), 128, 0, s>>>(B, m->h2, m->h1, a.d2, a.z1, 1, nullptr, gW2, gb2);
    k_back<<<nb(B * m->h1), 128, 0, s>>>(B, m->h2, m->h1, W2, a.d2, a.z1, a.d1);
    k_gw<<<nb(m->h1 * m->d_in + m->h1), 128, 0, s>>>(B, m->h1, m->d_in, a.d1, X, 0, m->d_norm, gW1, gb1);
    XB_LAUNCHED("mlp backward");
    return XB_OK;
}

}  // namespace

extern "C" {

int xb_mlp_create(int32_t d_in, int32_t h1, int32_t h2, int32_t nheads, const int32_t *heads,
                  uint64_t seed, xb_mlp **out) {
    if (!out || d_in < 1 || d_in > 16 || h1 < 1 || h2 < 1 || h1 > 1024 || h2 > 1024 || nheads < 1 ||
        nheads > 8 || !heads)
        return xb::set_error(XB_EINVAL, "mlp_create: bad dimensions");
    xb_mlp *m = new xb_mlp();
    m->d_in = d_in;
    m->h1 = h1;
    m->h2 = h2;
    m->nh = nheads;
    for (int h = 0; h < nheads; h++) {
        if (heads[h] < 2) {
            delete m;
            return xb::set_error(XB_EINVAL, "mlp_create: head %d has %d classes", h, heads[h]);
        }
        m->heads[h] = heads[h];
        m->o += heads[h];
    }
    m->np = (int64_t)h1 * d_in + h1 + (int64_t)h2 * h1 + h2 + (int64_t)m->o * h2 + m->o;
    // He-style initialisation on the host (seeded), biases zero
    std::vector<float> P(m->np, 0.f);
    std::mt19937_64 rng(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    auto fill = [&](int64_t off, int rows, int cols) {
        const float sc = std::sqrt(2.f / (float)cols);
        for (int64_t i = 0; i < (int64_t)rows * cols; i++) P[off + i] = nd(rng) * sc;
    };
    fill(0, h1, d_in);
    fill((int64_t)h1 * d_in + h1, h2, h1);
    fill((int64_t)h1 * d_in + h1 + (int64_t)h2 * h1 + h2, m->o, h2);
    std::vector<float> norm(2 * d_in);
    for (int i = 0; i < d_in; i++) {
        norm[i] = 0.f;
        norm[d_in + i] = 1.f;
    }
    m->h_mu.assign(d_in, 0.f);
    m->h_sd.assign(d_in, 1.f);
    cudaError_t e = cudaMalloc(&m->d_param, m->np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_grad, m->np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_m, m->np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_v, m->np * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_norm, 2 * d_in * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_heads, 8 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(m->d_param, P.data(), m->np * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->d_m, 0, m->np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->d_v, 0, m->np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(m->d_grad, 0, m->np * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(m->d_norm, norm.data(), norm.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->d_heads, m->heads, 8 * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        xb_mlp_destroy(m);
        return xb::cuda_error(e, "mlp_create");
    }
    *out = m;
    return XB_OK;
}

int xb_mlp_destroy(xb_mlp *m) {
    if (!m) return XB_OK;
    cudaDeviceSynchronize();
    cudaFree(m->d_param);
    cudaFree(m->d_grad);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    cudaFree(m->d_norm);
    cudaFree(m->d_heads);
    cudaFree(m->d_act);
    cudaFree(m->d_loss);
    cudaFree(m->d_xb);
    cudaFree(m->d_lb);
    cudaFree(m->d_idx);
    delete m;
    return XB_OK;
}

int64_t xb_mlp_param_count(const xb_mlp *m) { return m ? m->np : -1; }

int xb_mlp_get_params(const xb_mlp *m, float *host) {
    if (!m || !host) return xb::set_error(XB_EINVAL, "mlp_get_params: NULL");
    XB_CUDA(cudaMemcpy(host, m->d_param, m->np * sizeof(float), cudaMemcpyDeviceToHost));
    return XB_OK;
}

int xb_mlp_set_params(xb_mlp *m, const float *host) {
    if (!m || !host) return xb::set_error(XB_EINVAL, "mlp_set_params: NULL");
    XB_CUDA(cudaMemcpy(m->d_param, host, m->np * sizeof(float), cudaMemcpyHostToDevice));
    return XB_OK;
}

int xb_mlp_set_norm(xb_mlp *m, const float *mu, const float *sd) {
    if (!m || !mu || !sd) return xb::set_error(XB_EINVAL, "mlp_set_norm: NULL");
    std::vector<float> norm(2 * m->d_in);
    for (int i = 0; i < m->d_in; i++) {
        if (!(sd[i] > 0.f)) return xb::set_error(XB_EINVAL, "mlp_set_norm: sd[%d] <= 0", i);
        norm[i] = mu[i];
        norm[m->d_in + i] = sd[i];
    }
    m->h_mu.assign(mu, mu + m->d_in);
    m->h_sd.assign(sd, sd + m->d_in);
    XB_CUDA(cudaMemcpy(m->d_norm, norm.data(), norm.size() * sizeof(float), cudaMemcpyHostToDevice));
    return XB_OK;
}

int xb_mlp_forward(xb_mlp *m, const float *X, int32_t B, float *logits, void *stream) {
    if (!m || B < 0 || (B > 0 && (!X || !logits))) return xb::set_error(XB_EINVAL, "mlp_forward: bad argument");
    if (B == 0) return XB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    XB_TRY(forward(m, X, B, s));
    XB_CUDA(cudaMemcpyAsync(logits, act_of(m).lg, (size_t)B * m->o * sizeof(float),
                            cudaMemcpyDeviceToDevice, s));
    return XB_OK;
}

int xb_mlp_loss_grad(xb_mlp *m, const float *X, const int32_t *labels, int32_t B, float *loss,
                     float *grad_out, void *stream) {
    if (!m || B < 1 || !X || !labels) return xb::set_error(XB_EINVAL, "mlp_loss_grad: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    XB_TRY(ensure_act(m, B));
    XB_TRY(loss_grad(m, X, labels, B, m->d_loss + m->act_cap, s));
    if (grad_out)
        XB_CUDA(cudaMemcpyAsync(grad_out, m->d_grad, m->np * sizeof(float), cudaMemcpyDeviceToDevice, s));
    float l = 0.f;
    XB_CUDA(cudaMemcpyAsync(&l, m->d_loss + m->act_cap, sizeof(float), cudaMemcpyDeviceToHost, s));
    XB_CUDA(cudaStreamSynchronize(s));
    if (loss) *loss = l;
    return XB_OK;
}

int xb_mlp_adam(xb_mlp *m, int32_t t, float lr, float b1, float b2, float eps, void *stream) {
    if (!m || t < 1) return xb::set_error(XB_EINVAL, "mlp_adam: bad argument");
    const float c1 = 1.f - std::pow(b1, (float)t), c2 = 1.f - std::pow(b2, (float)t);
    k_adam<<<std::max<int64_t>(1, std::min<int64_t>((m->np + 255) / 256, 1024)), 256, 0,
             (cudaStream_t)stream>>>(m->np, m->d_param, m->d_grad, m->d_m, m->d_v, lr, b1, b2, eps,
                                     c1, c2);
    XB_LAUNCHED("k_adam");
    return XB_OK;
}

int xb_mlp_train(xb_mlp *m, const float *X, const int32_t *labels, int32_t N, int32_t epochs,
                 int32_t batch, float lr, uint64_t seed, float *final_loss, void *stream) {
    if (!m || N < 1 || !X || !labels || epochs < 0 || batch < 1)
        return xb::set_error(XB_EINVAL, "mlp_train: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    batch = std::min(batch, N);
    if ((size_t)batch > m->mb_cap) {
        cudaFree(m->d_xb);
        cudaFree(m->d_lb);
        cudaFree(m->d_idx);
        m->d_xb = nullptr;
        m->d_lb = nullptr;
        m->d_idx = nullptr;
        XB_CUDA(cudaMalloc(&m->d_xb, (size_t)batch * m->d_in * sizeof(float)));
        XB_CUDA(cudaMalloc(&m->d_lb, (size_t)batch * m->nh * sizeof(int)));
        XB_CUDA(cudaMalloc(&m->d_idx, (size_t)N * sizeof(int)));
        m->mb_cap = batch;
    }
    int *d_perm = nullptr;
    XB_CUDA(cudaMalloc(&d_perm, (size_t)N * sizeof(int)));
    XB_TRY(ensure_act(m, std::max(batch, N)));
    std::vector<int> perm(N);
    for (int i = 0; i < N; i++) perm[i] = i;
    std::mt19937_64 rng(seed);
    int t = 0;
    for (int ep = 0; ep < epochs; ep++) {
        std::shuffle(perm.begin(), perm.end(), rng);
        cudaMemcpyAsync(d_perm, perm.data(), (size_t)N * sizeof(int), cudaMemcpyHostToDevice, s);
        for (int b0 = 0; b0 < N; b0 += batch) {
            const int B = std::min(batch, N - b0);
            k_gather_rows<<<(B + 127) / 128, 128, 0, s>>>(B, m->d_in, d_perm + b0, X, m->d_xb,
                                                           labels, m->nh, m->d_lb);
            int r = loss_grad(m, m->d_xb, m->d_lb, B, m->d_loss + m->act_cap, s);
            if (r == XB_OK) r = xb_mlp_adam(m, ++t, lr, 0.9f, 0.999f, 1e-8f, s);
            if (r != XB_OK) {
                cudaFree(d_perm);
                return r;
            }
        }
        cudaStreamSynchronize(s);  // the host permutation buffer is reused
    }
    cudaFree(d_perm);
    if (final_loss) {
        float l = 0.f;
        XB_TRY(loss_grad(m, X, labels, N, m->d_loss + m->act_cap, s));
        XB_CUDA(cudaMemcpyAsync(&l, m->d_loss + m->act_cap, sizeof(float), cudaMemcpyDeviceToHost, s));
        XB_CUDA(cudaStreamSynchronize(s));
        *final_loss = l;
    }
    return XB_OK;
}

int xb_mlp_predict(xb_mlp *m, const float *X, int32_t B, int32_t *out_host, void *stream) {
    if (!m || B < 0 || (B > 0 && (!X || !out_host))) return xb::set_error(XB_EINVAL, "mlp_predict: bad argument");
    if (B == 0) return XB_OK;
    cudaStream_t s = (cudaStream_t)stream;
    XB_TRY(forward(m, X, B, s));
    int *d_out = nullptr;
    XB_CUDA(cudaMalloc(&d_out, (size_t)B * m->nh * sizeof(int)));
    k_argmax<<<(B + 127) / 128, 128, 0, s>>>(B, dims_of(m), m->d_heads, act_of(m).lg, d_out);
    cudaError_t e = cudaMemcpyAsync(out_host, d_out, (size_t)B * m->nh * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_out);
    if (e != cudaSuccess) return xb::cuda_error(e, "mlp_predict");
    return XB_OK;
}

// File: "XBMLP001", int32 d_in,h1,h2,nh, heads[8], float mu[d_in], sd[d_in], float P[np].
int xb_mlp_save(const xb_mlp *m, const char *path) {
    if (!m || !path) return xb::set_error(XB_EINVAL, "mlp_save: NULL");
    std::vector<float> P(m->np);
    XB_CUDA(cudaMemcpy(P.data(), m->d_param, m->np * sizeof(float), cudaMemcpyDeviceToHost));
    FILE *f = std::fopen(path, "wb");
    if (!f) return xb::set_error(XB_EINVAL, "mlp_save: cannot open %s", path);
    const int32_t hdr[4] = {m->d_in, m->h1, m->h2, m->nh};
    bool ok = std::fwrite("XBMLP001", 1, 8, f) == 8 && std::fwrite(hdr, 4, 4, f) == 4 &&
              std::fwrite(m->heads, 4, 8, f) == 8 &&
              std::fwrite(m->h_mu.data(), 4, m->d_in, f) == (size_t)m->d_in &&
              std::fwrite(m->h_sd.data(), 4, m->d_in, f) == (size_t)m->d_in &&
              std::fwrite(P.data(), 4, m->np, f) == (size_t)m->np;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? XB_OK : xb::set_error(XB_EINVAL, "mlp_save: write failed");
}

int xb_mlp_load(const char *path, xb_mlp **out) {
    if (!path || !out) return xb::set_error(XB_EINVAL, "mlp_load: NULL");
    FILE *f = std::fopen(path, "rb");
    if (!f) return xb::set_error(XB_EINVAL, "mlp_load: cannot open %s", path);
    char magic[8];
    int32_t hdr[4], heads[8];
    if (std::fread(magic, 1, 8, f) != 8 || std::memcmp(magic, "XBMLP001", 8) != 0 ||
        std::fread(hdr, 4, 4, f) != 4 || std::fread(heads, 4, 8, f) != 8) {
        std::fclose(f);
        return xb::set_error(XB_EINVAL, "mlp_load: bad header in %s", path);
    }
    xb_mlp *m = nullptr;
    int r = xb_mlp_create(hdr[0], hdr[1], hdr[2], hdr[3], heads, 0, &m);
    if (r != XB_OK) {
        std::fclose(f);
        return r;
    }
    std::vector<float> mu(m->d_in), sd(m->d_in), P(m->np);
    const bool ok = std::fread(mu.data(), 4, m->d_in, f) == (size_t)m->d_in &&
                    std::fread(sd.data(), 4, m->d_in, f) == (size_t)m->d_in &&
                    std::fread(P.data(), 4, m->np, f) == (size_t)m->np;
    std::fclose(f);
    if (!ok) {
        xb_mlp_destroy(m);
        return xb::set_error(XB_EINVAL, "mlp_load: truncated %s", path);
    }
    r = xb_mlp_set_norm(m, mu.data(), sd.data());
    if (r == XB_OK) r = xb_mlp_set_params(m, P.data());
    if (r != XB_OK) {
        xb_mlp_destroy(m);
        return r;
    }
    *out = m;
    return XB_OK;
}

}  // extern "C"
