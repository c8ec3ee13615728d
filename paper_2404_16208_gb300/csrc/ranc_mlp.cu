// Design-space surrogate: forward, MSE backward and Adam for a small fully
// connected network (see include/ranc_mlp.h).  bf16 weights in the passes,
// fp32 accumulation, fp32 masters and optimizer state.  Every matrix product
// (forward, gradient of the inputs, gradient of the weights) runs on the
// tensor cores with mma.sync.m16n8k16 bf16 -> fp32: an fp32 operand enters as
// two bf16 terms x = hi + lo (hi = bf16(x), lo = bf16(x - hi): 16 significant
// bits), a product of two such operands as hi*hi + hi*lo + lo*hi; bf16
// weights enter exactly.  Tiles and the order of the sums are fixed, so the
// results are deterministic.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
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

// ---------------------------------------------------------------------------
// Tensor-core GEMM: C[m][n] = sum_k A(m, k) * B(n, k) for the three products
// of a layer, with strided operands (element (m, k) of A at A[m * am + k * ak],
// element (n, k) of B at B[n * bn + k * bk]).  A CTA (4 warps) computes a 64 x
// 64 tile of C over K-tiles of 32: the operands are staged in shared memory as
// bf16 (hi and lo terms of fp32 operands), each warp holds a 32 x 32 block as
// 2 x 4 m16n8 accumulators and issues mma.sync.m16n8k16 per K-step.
// ---------------------------------------------------------------------------

constexpr int kGM = 64, kGN = 64, kGK = 32, kGPad = 40;  // tile sizes; shared rows of 40 bf16 (no bank conflicts)

enum { kEpiForward = 0, kEpiMaskRelu = 1, kEpiStore = 2 };

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <typename T>
__device__ __forceinline__ float as_f32(T x) {
    if constexpr (std::is_same<T, float>::value) return x;
    else return __bfloat162float(x);
}

// Epilogues: forward (C + bias -> Z, relu or identity -> Act), gradient of
// the inputs (C * (Z > 0)), plain store.
template <typename TB, bool kSplitB, int kEpi>
__global__ void __launch_bounds__(128) gemm_tc(int M, int N, int K, const float *A, long long am, long long ak, const TB *B,
                                               long long bn, long long bk, float *C, const float *bias, int relu,
                                               float *Act, const float *Zmask) {
    __shared__ __align__(16) __nv_bfloat16 sa[2][kGM][kGPad], sb[2][kGN][kGPad];  // [hi / lo][row][k]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, tq = lane & 3;
    const int m0 = blockIdx.y * kGM, n0 = blockIdx.x * kGN;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    for (int k0 = 0; k0 < K; k0 += kGK) {
        for (int idx = tid; idx < kGM * kGK; idx += 128) {
            const int r = idx / kGK, kk = idx % kGK, m = m0 + r, k = k0 + kk;
            const float x = (m < M && k < K) ? A[(long long)m * am + (long long)k * ak] : 0.f;
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            sa[0][r][kk] = hi;
            sa[1][r][kk] = __float2bfloat16_rn(x - __bfloat162float(hi));
        }
        for (int idx = tid; idx < kGN * kGK; idx += 128) {
            const int r = idx / kGK, kk = idx % kGK, n = n0 + r, k = k0 + kk;
            const float x = (n < N && k < K) ? as_f32(B[(long long)n * bn + (long long)k * bk]) : 0.f;
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            sb[0][r][kk] = hi;
            if constexpr (kSplitB) sb[1][r][kk] = __float2bfloat16_rn(x - __bfloat162float(hi));
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kGK; ks += 16) {
            uint32_t af[2][2][4], bf[2][4][2];  // [hi / lo][tile][regs]
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int r = wm + 16 * i + g;
                    af[h][i][0] = *reinterpret_cast<const uint32_t *>(&sa[h][r][ks + 2 * tq]);
                    af[h][i][1] = *reinterpret_cast<const uint32_t *>(&sa[h][r + 8][ks + 2 * tq]);
                    af[h][i][2] = *reinterpret_cast<const uint32_t *>(&sa[h][r][ks + 2 * tq + 8]);
                    af[h][i][3] = *reinterpret_cast<const uint32_t *>(&sa[h][r + 8][ks + 2 * tq + 8]);
                }
                if (h == 1 && !kSplitB) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = wn + 8 * j + g;
                    bf[h][j][0] = *reinterpret_cast<const uint32_t *>(&sb[h][r][ks + 2 * tq]);
                    bf[h][j][1] = *reinterpret_cast<const uint32_t *>(&sb[h][r][ks + 2 * tq + 8]);
                }
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    mma_bf16(acc[i][j], af[0][i][0], af[0][i][1], af[0][i][2], af[0][i][3], bf[0][j][0], bf[0][j][1]);
                    mma_bf16(acc[i][j], af[1][i][0], af[1][i][1], af[1][i][2], af[1][i][3], bf[0][j][0], bf[0][j][1]);
                    if constexpr (kSplitB)
                        mma_bf16(acc[i][j], af[0][i][0], af[0][i][1], af[0][i][2], af[0][i][3], bf[1][j][0], bf[1][j][1]);
                }
        }
        __syncthreads();
    }
    // accumulator element e of tile (i, j): row wm + 16 i + g + 8 (e / 2), column wn + 8 j + 2 tq + e % 2
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + 16 * i + g + 8 * (e >> 1), n = n0 + wn + 8 * j + 2 * tq + (e & 1);
                if (m >= M || n >= N) continue;
                const size_t o = (size_t)m * N + n;
                float v = acc[i][j][e];
                if constexpr (kEpi == kEpiForward) {
                    v += bias[n];
                    C[o] = v;
                    Act[o] = relu ? fmaxf(v, 0.f) : v;
                } else if constexpr (kEpi == kEpiMaskRelu) {
                    C[o] = Zmask[o] > 0.f ? v : 0.f;
                } else {
                    C[o] = v;
                }
            }
}

dim3 gemm_grid(int M, int N) { return dim3((N + kGN - 1) / kGN, (M + kGM - 1) / kGM); }

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

// db[o] = sum_b dZ[b][o] (fixed order).
__global__ void bias_grad(const float *dZ, int batch, int out, float *db) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= out) return;
    float acc = 0.f;
    for (int b = 0; b < batch; ++b) acc += dZ[(size_t)b * out + o];
    db[o] = acc;
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
        // Z[b][o] = sum_i X[b][i] W[o][i] + bias[o]
        gemm_tc<__nv_bfloat16, false, kEpiForward><<<gemm_grid(batch, L.out), 128, 0, m->stream>>>(
            batch, L.out, L.in, in, L.in, 1, m->w16 + L.w_off, L.in, 1, m->Z[l], m->p + L.b_off, l + 1 < m->n_layers,
            m->A[l], nullptr);
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
        // dW[o][i] = sum_b dZ[b][o] Xin[b][i]: A(o, b) = dZ[b][o], B(i, b) = Xin[b][i]
        gemm_tc<float, true, kEpiStore><<<gemm_grid(L.out, L.in), 128, 0, m->stream>>>(
            L.out, L.in, batch, dz, 1, L.out, xin, 1, L.in, m->g + L.w_off, nullptr, 0, nullptr, nullptr);
        MLP_CUDA(m, cudaGetLastError());
        bias_grad<<<(L.out + 127) / 128, 128, 0, m->stream>>>(dz, batch, L.out, m->g + L.b_off);
        MLP_CUDA(m, cudaGetLastError());
        if (l > 0) {
            // dZprev[b][i] = (sum_o dZ[b][o] W[o][i]) (Zprev[b][i] > 0): A(b, o) = dZ[b][o], B(i, o) = W[o][i]
            gemm_tc<__nv_bfloat16, false, kEpiMaskRelu><<<gemm_grid(batch, L.in), 128, 0, m->stream>>>(
                batch, L.in, L.out, dz, L.out, 1, m->w16 + L.w_off, 1, L.in, dz_prev, nullptr, 0, nullptr, m->Z[l - 1]);
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
