// Design-space surrogate: forward, MSE backward and Adam for a small fully
// connected network (see include/ranc_mlp.h).  bf16 weights in the passes,
// fp32 accumulation, fp32 masters and optimizer state.  The layers are at most
// 1024 wide and the batches a few hundred rows, so each kernel maps one thread
// to one output element and sums in a fixed order (deterministic results).

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "ranc.h"
#include "ranc_internal.cuh"
#include "ranc_mlp.h"

namespace {

struct Layer {
    int in = 0, out = 0;
    size_t w_off = 0, b_off = 0;  // offsets into the flat parameter arrays
};

}  // namespace

struct ranc_mlp {
    int n_layers = 0, max_batch = 0;
    std::vector<Layer> layers;
    size_t n_params = 0;
    cudaStream_t stream = nullptr;
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;  // masters, grads, Adam moments
    __nv_bfloat16 *w16 = nullptr;                                   // bf16 weights (same offsets)
    char *is_w = nullptr;                                            // 1 for weight entries, 0 for biases
    std::vector<float *> Z, A;                                      // per layer [max_batch][out]
    float *dz0 = nullptr, *dz1 = nullptr;                            // ping-pong [max_batch][max_dim]
    float *loss = nullptr;
    long long step = 0;
    std::string err;
};

namespace {

int mlp_fail(ranc_mlp *m, int code, const char *fmt, ...) {
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (m) m->err = buf;
    return code;
}

thread_local std::string g_mlp_create_error;

#define MLP_CUDA(m, expr)                                                                        \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) return mlp_fail((m), RANC_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

// Z = X W^T + b (and A = relu(Z) when relu), one thread per output element.
__global__ void linear_fwd(const float *X, const __nv_bfloat16 *W, const float *bias, int batch, int in, int out,
                           int relu, float *Z, float *A) {
    extern __shared__ float xs[];
    const int b = blockIdx.y;
    for (int i = threadIdx.x; i < in; i += blockDim.x) xs[i] = X[(size_t)b * in + i];
    __syncthreads();
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= out || b >= batch) return;
    const __nv_bfloat16 *w = W + (size_t)o * in;
    float acc = bias[o];
    for (int i = 0; i < in; ++i) acc = fmaf(xs[i], __bfloat162float(w[i]), acc);
    Z[(size_t)b * out + o] = acc;
    A[(size_t)b * out + o] = relu ? fmaxf(acc, 0.f) : acc;
}

// dY = 2 (y - t) / (batch * d); loss = mean (y - t)^2 summed per row then over rows.
__global__ void mse_grad(const float *Y, const float *T, int batch, int d, float *dY, float *row_loss) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const float scale = 2.f / ((float)batch * (float)d);
    float s = 0.f;
    for (int k = 0; k < d; ++k) {
        const float e = Y[(size_t)b * d + k] - T[(size_t)b * d + k];
        dY[(size_t)b * d + k] = scale * e;
        s += e * e;
    }
    row_loss[b] = s / ((float)batch * (float)d);
}

__global__ void sum_rows(const float *row_loss, int batch, float *loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        float s = 0.f;
        for (int b = 0; b < batch; ++b) s += row_loss[b];
        *loss = s;
    }
}

// dW[o][i] = sum_b dZ[b][o] * Xin[b][i];  db[o] = sum_b dZ[b][o].
__global__ void linear_bwd_weight(const float *dZ, const float *Xin, int batch, int in, int out, float *dW,
                                  float *db) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < out * in) {
        const int o = idx / in, i = idx % in;
        float acc = 0.f;
        for (int b = 0; b < batch; ++b) acc = fmaf(dZ[(size_t)b * out + o], Xin[(size_t)b * in + i], acc);
        dW[idx] = acc;
    }
    if (idx < out) {
        float acc = 0.f;
        for (int b = 0; b < batch; ++b) acc += dZ[(size_t)b * out + idx];
        db[idx] = acc;
    }
}

// dZprev[b][i] = (sum_o dZ[b][o] * W[o][i]) * (Zprev[b][i] > 0).
__global__ void linear_bwd_data(const float *dZ, const __nv_bfloat16 *W, const float *Zprev, int batch, int in,
                                int out, float *dZprev) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= batch * in) return;
    const int b = idx / in, i = idx % in;
    float acc = 0.f;
    for (int o = 0; o < out; ++o) acc = fmaf(dZ[(size_t)b * out + o], __bfloat162float(W[(size_t)o * in + i]), acc);
    dZprev[idx] = Zprev[idx] > 0.f ? acc : 0.f;
}

__global__ void adam_kernel(float *p, const float *g, float *m1, float *m2, __nv_bfloat16 *w16, const char *is_w,
                            size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float a = b1 * m1[k] + (1.f - b1) * gk;
        const float v = b2 * m2[k] + (1.f - b2) * gk * gk;
        m1[k] = a;
        m2[k] = v;
        const float pk = p[k] - lr * (a / c1) / (sqrtf(v / c2) + eps);
        p[k] = pk;
        if (is_w[k]) w16[k] = __float2bfloat16_rn(pk);
    }
}

__global__ void to_bf16(const float *p, __nv_bfloat16 *w16, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        w16[k] = __float2bfloat16_rn(p[k]);
}

__global__ void bf16_to_f32(const __nv_bfloat16 *w16, float *out, size_t n) {
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        out[k] = __bfloat162float(w16[k]);
}

void mlp_free(ranc_mlp *m) {
    void *ptrs[] = {m->p, m->g, m->m1, m->m2, m->w16, m->dz0, m->dz1, m->loss, m->is_w};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    for (float *q : m->Z) cudaFree(q);
    for (float *q : m->A) cudaFree(q);
}

// Marks which flat entries are weights (bf16 copies) rather than biases.
char *make_is_w(ranc_mlp *m) {
    std::vector<char> h(m->n_params, 0);
    for (const Layer &L : m->layers)
        for (size_t k = 0; k < (size_t)L.in * L.out; ++k) h[L.w_off + k] = 1;
    char *d = nullptr;
    if (ranc::dev_alloc((void **)&d, h.size()) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, h.data(), h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    return d;
}

int mlp_forward(ranc_mlp *m, const float *x, int batch) {
    const float *in = x;
    for (int l = 0; l < m->n_layers; ++l) {
        const Layer &L = m->layers[l];
        dim3 grid((L.out + 127) / 128, batch);
        linear_fwd<<<grid, 128, L.in * sizeof(float), m->stream>>>(in, m->w16 + L.w_off, m->p + L.b_off, batch, L.in,
                                                                   L.out, l + 1 < m->n_layers, m->Z[l], m->A[l]);
        MLP_CUDA(m, cudaGetLastError());
        in = m->A[l];
    }
    return RANC_OK;
}

}  // namespace

extern "C" int ranc_mlp_create(int32_t n_layers, const int32_t *dims, int32_t max_batch, uint64_t seed,
                               void *cuda_stream, ranc_mlp **out) {
    if (!out) return RANC_EINVAL;
    *out = nullptr;
    if (n_layers < 1 || !dims || max_batch < 1) {
        g_mlp_create_error = "n_layers >= 1, dims and max_batch >= 1 are required";
        return RANC_EINVAL;
    }
    for (int l = 0; l <= n_layers; ++l)
        if (dims[l] < 1 || dims[l] > 1024) {
            g_mlp_create_error = "every layer width must lie in [1, 1024]";
            return RANC_EINVAL;
        }
    ranc_mlp *m = new (std::nothrow) ranc_mlp();
    if (!m) return RANC_ENOMEM;
    m->n_layers = n_layers;
    m->max_batch = max_batch;
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    size_t off = 0;
    int max_dim = 0;
    for (int l = 0; l < n_layers; ++l) {
        Layer L;
        L.in = dims[l];
        L.out = dims[l + 1];
        L.w_off = off;
        off += (size_t)L.in * L.out;
        L.b_off = off;
        off += L.out;
        m->layers.push_back(L);
        max_dim = std::max(max_dim, std::max(L.in, L.out));
    }
    m->n_params = off;
    // Initial weights: uniform in +-sqrt(6 / fan_in) from SplitMix64 draws.
    std::vector<float> h(off, 0.f);
    uint64_t state = seed;
    for (const Layer &L : m->layers) {
        const float lim = sqrtf(6.f / (float)L.in);
        for (size_t k = 0; k < (size_t)L.in * L.out; ++k) {
            state += 0x9E3779B97F4A7C15ull;
            uint64_t z = state;
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            const float u = (float)((z >> 40) * (1.0 / 16777216.0));
            h[L.w_off + k] = (2.f * u - 1.f) * lim;
        }
    }
    auto fail_create = [&](int code, const char *msg) {
        g_mlp_create_error = msg;
        mlp_free(m);
        delete m;
        return code;
    };
    const size_t act = (size_t)max_batch * max_dim;
    if (ranc::dev_alloc((void **)&m->p, off * 4) != cudaSuccess || ranc::dev_alloc((void **)&m->g, off * 4) != cudaSuccess ||
        ranc::dev_alloc((void **)&m->m1, off * 4) != cudaSuccess ||
        ranc::dev_alloc((void **)&m->m2, off * 4) != cudaSuccess ||
        ranc::dev_alloc((void **)&m->w16, off * 2) != cudaSuccess ||
        ranc::dev_alloc((void **)&m->dz0, act * 4) != cudaSuccess ||
        ranc::dev_alloc((void **)&m->dz1, act * 4) != cudaSuccess ||
        ranc::dev_alloc((void **)&m->loss, ((size_t)max_batch + 1) * 4) != cudaSuccess)
        return fail_create(RANC_ENOMEM, "device allocation");
    for (int l = 0; l < n_layers; ++l) {
        float *z = nullptr, *a = nullptr;
        const size_t n = (size_t)max_batch * m->layers[l].out * 4;
        if (ranc::dev_alloc((void **)&z, n) != cudaSuccess || ranc::dev_alloc((void **)&a, n) != cudaSuccess) {
            if (z) cudaFree(z);
            return fail_create(RANC_ENOMEM, "device allocation of activations");
        }
        m->Z.push_back(z);
        m->A.push_back(a);
    }
    if (!(m->is_w = make_is_w(m))) return fail_create(RANC_ENOMEM, "device allocation of the weight mask");
    *out = m;
    int rc = ranc_mlp_set_params(m, h.data());
    if (rc != RANC_OK) {
        *out = nullptr;
        return fail_create(rc, "initial parameter upload");
    }
    return RANC_OK;
}

extern "C" int ranc_mlp_param_count(const ranc_mlp *m, int64_t *count) {
    if (!m || !count) return RANC_EINVAL;
    *count = (int64_t)m->n_params;
    return RANC_OK;
}

extern "C" int ranc_mlp_set_params(ranc_mlp *m, const float *params) {
    if (!m || !params) return RANC_EINVAL;
    MLP_CUDA(m, cudaMemcpyAsync(m->p, params, m->n_params * 4, cudaMemcpyHostToDevice, m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->m1, 0, m->n_params * 4, m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->m2, 0, m->n_params * 4, m->stream));
    to_bf16<<<256, 256, 0, m->stream>>>(m->p, m->w16, m->n_params);
    MLP_CUDA(m, cudaGetLastError());
    m->step = 0;
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return RANC_OK;
}

extern "C" int ranc_mlp_get_params(ranc_mlp *m, float *params) {
    if (!m || !params) return RANC_EINVAL;
    std::vector<float> h(m->n_params);
    float *d = nullptr;
    if (ranc::dev_alloc((void **)&d, m->n_params * 4) != cudaSuccess) return mlp_fail(m, RANC_ENOMEM, "scratch");
    bf16_to_f32<<<256, 256, 0, m->stream>>>(m->w16, d, m->n_params);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, m->n_params * 4, cudaMemcpyDeviceToHost, m->stream);
    std::vector<float> hp(m->n_params);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), m->p, m->n_params * 4, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    cudaFree(d);
    if (e != cudaSuccess) return mlp_fail(m, RANC_ECUDA, "%s", cudaGetErrorString(e));
    for (const Layer &L : m->layers) {
        memcpy(params + L.w_off, h.data() + L.w_off, (size_t)L.in * L.out * 4);
        memcpy(params + L.b_off, hp.data() + L.b_off, (size_t)L.out * 4);
    }
    return RANC_OK;
}

extern "C" int ranc_mlp_forward(ranc_mlp *m, const float *x, int32_t batch, float *y) {
    if (!m || !x || !y || batch < 1 || batch > m->max_batch) return mlp_fail(m, RANC_EINVAL, "bad forward arguments");
    int rc = mlp_forward(m, x, batch);
    if (rc) return rc;
    const Layer &L = m->layers.back();
    MLP_CUDA(m, cudaMemcpyAsync(y, m->A.back(), (size_t)batch * L.out * 4, cudaMemcpyDeviceToDevice, m->stream));
    return RANC_OK;
}

extern "C" int ranc_mlp_loss_backward(ranc_mlp *m, const float *x, const float *target, int32_t batch, float *loss,
                                      float *grads) {
    if (!m || !x || !target || batch < 1 || batch > m->max_batch)
        return mlp_fail(m, RANC_EINVAL, "bad backward arguments");
    int rc = mlp_forward(m, x, batch);
    if (rc) return rc;
    const int L_last = m->n_layers - 1;
    const int d_out = m->layers[L_last].out;
    mse_grad<<<(batch + 127) / 128, 128, 0, m->stream>>>(m->A[L_last], target, batch, d_out, m->dz0, m->loss + 1);
    MLP_CUDA(m, cudaGetLastError());
    sum_rows<<<1, 32, 0, m->stream>>>(m->loss + 1, batch, m->loss);
    MLP_CUDA(m, cudaGetLastError());
    float *dz = m->dz0, *dz_prev = m->dz1;
    for (int l = L_last; l >= 0; --l) {
        const Layer &L = m->layers[l];
        const float *xin = l > 0 ? m->A[l - 1] : x;
        const int nw = L.in * L.out;
        linear_bwd_weight<<<(nw + 255) / 256, 256, 0, m->stream>>>(dz, xin, batch, L.in, L.out, m->g + L.w_off,
                                                                   m->g + L.b_off);
        MLP_CUDA(m, cudaGetLastError());
        if (l > 0) {
            linear_bwd_data<<<(batch * L.in + 255) / 256, 256, 0, m->stream>>>(dz, m->w16 + L.w_off, m->Z[l - 1],
                                                                               batch, L.in, L.out, dz_prev);
            MLP_CUDA(m, cudaGetLastError());
            std::swap(dz, dz_prev);
        }
    }
    if (loss) MLP_CUDA(m, cudaMemcpyAsync(loss, m->loss, 4, cudaMemcpyDeviceToHost, m->stream));
    if (grads) MLP_CUDA(m, cudaMemcpyAsync(grads, m->g, m->n_params * 4, cudaMemcpyDeviceToHost, m->stream));
    if (loss || grads) MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return RANC_OK;
}

extern "C" int ranc_mlp_adam_step(ranc_mlp *m, float lr, float beta1, float beta2, float eps) {
    if (!m) return RANC_EINVAL;
    m->step++;
    const float c1 = 1.f - powf(beta1, (float)m->step), c2 = 1.f - powf(beta2, (float)m->step);
    adam_kernel<<<256, 256, 0, m->stream>>>(m->p, m->g, m->m1, m->m2, m->w16, m->is_w, m->n_params, lr, beta1, beta2, eps,
                                            c1, c2);
    MLP_CUDA(m, cudaGetLastError());
    return RANC_OK;
}

extern "C" void ranc_mlp_destroy(ranc_mlp *m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    mlp_free(m);
    delete m;
}

extern "C" const char *ranc_mlp_last_error(const ranc_mlp *m) {
    if (!m) return g_mlp_create_error.c_str();
    return m->err.c_str();
}
