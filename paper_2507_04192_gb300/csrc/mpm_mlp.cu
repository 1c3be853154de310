// Small fully connected network trained and evaluated on the tcgen05 tensor
// cores: the learned warm start of the basal-friction inversion (a map from
// tracked-particle observations to per-segment friction coefficients).
//
// Layers: z_l = x_l W_l^T + b_l, x_{l+1} = GELU(z_l) (exact erf form) or
// max(z_l, 0) for the hidden layers, output y = lo + (hi - lo) sigmoid(z_last)
// or y = z_last (the coordinate network of Eq. nn_apprx).  Weights are kept in
// fp32 (Adam state too) with bf16 copies (and their transposes) as GEMM
// operands; activations and back-propagated gradients enter the GEMMs as bf16
// and every GEMM accumulates in fp32 in TMEM.  Loss: mean squared error.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mpm.h"
#include "mpm_umma.cuh"

using namespace mpm;

namespace {

__global__ void k_f32_to_bf16(const float *__restrict__ in, __nv_bfloat16 *__restrict__ out, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(in[i]);
}

// out[c][r] = in[r][c] (rows x cols -> cols x rows), bf16.
__global__ void k_transpose_bf16(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out, int rows,
                                 int cols)
{
    __shared__ __nv_bfloat16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = r0 + j, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[j][threadIdx.x] = in[(int64_t)r * cols + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int c = c0 + j, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[(int64_t)c * rows + r] = tile[threadIdx.x][j];
    }
}

__device__ __forceinline__ float gelu_grad_f(float z)
{
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Loss and output gradient: L = mean (y - t)^2; dz = dL/dy (hi - lo) s (1 - s)
// (dz = dL/dy for the linear output).
__global__ void k_mse_out(const float *__restrict__ y, const float *__restrict__ t, const float *__restrict__ z,
                          float *__restrict__ dz, int64_t n, float lo, float hi, double *__restrict__ loss,
                          int linear)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float e = y[i] - t[i];
        acc += (double)e * e;
        if (linear) {
            dz[i] = 2.0f * e / (float)n;
        } else {
            const float s = 1.0f / (1.0f + expf(-z[i]));
            dz[i] = 2.0f * e / (float)n * (hi - lo) * s * (1.0f - s);
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc / (double)n);
}

// dz_prev = da * GELU'(z_prev), or da * [z_prev > 0] for ReLU.
__global__ void k_act_back(const float *__restrict__ da, const float *__restrict__ z, float *__restrict__ dz,
                           int64_t n, int relu)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dz[i] = relu ? (z[i] > 0.0f ? da[i] : 0.0f) : da[i] * gelu_grad_f(z[i]);
}

// Output gradient from a given dL/dy: dz = dy (hi - lo) s (1 - s) for the scaled
// sigmoid, dz = dy for the linear output.
__global__ void k_out_back(const float *__restrict__ dy, const float *__restrict__ z, float *__restrict__ dz,
                           int64_t n, float lo, float hi, int linear)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (linear) {
            dz[i] = dy[i];
        } else {
            const float s = 1.0f / (1.0f + expf(-z[i]));
            dz[i] = dy[i] * (hi - lo) * s * (1.0f - s);
        }
    }
}

// db[c] = sum_r dz[r][c].
__global__ void k_col_sum(const float *__restrict__ dz, float *__restrict__ db, int rows, int cols)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dz[(int64_t)r * cols + c];
    db[c] = s;
}

// Adam on fp32 master parameters (bias-corrected moments).
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

int blocks_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

}  // namespace

struct mpm_mlp {
    int L = 0, max_batch = 0;
    std::vector<int> w;                           // widths, L + 1
    float lo = 0.f, hi = 1.f;
    int hidden_act = MPM_ACT_GELU, out_act = MPM_OUT_SIGMOID;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<float *> W, b, gW, gb, mW, vW, mb, vb;     // fp32
    std::vector<__nv_bfloat16 *> Wb, WbT;                   // bf16 weight copies
    std::vector<__nv_bfloat16 *> X, XT;                     // layer inputs (bf16) and transposes, l = 0..L-1
    std::vector<float *> Z, dZ;                             // pre-activations and their gradients (fp32)
    std::vector<__nv_bfloat16 *> dZb, dZbT;
    float *Y = nullptr, *T = nullptr, *dA = nullptr, *X0f = nullptr;
    double *loss = nullptr;
    int32_t *status = nullptr;
    int64_t step = 0;
    std::string err;
};

namespace {

template <class T> int malloc_n(mpm_mlp *m, T **p, size_t count)
{
    if (cudaMalloc((void **)p, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
        cudaGetLastError();
        m->err = "cudaMalloc failed";
        return MPM_ENOMEM;
    }
    return MPM_OK;
}

void refresh_bf16(mpm_mlp *m, int l)
{
    const int64_t n = (int64_t)m->w[l + 1] * m->w[l];
    k_f32_to_bf16<<<blocks_for(n), 256, 0, m->stream>>>(m->W[l], m->Wb[l], n);
    dim3 tb(32, 8), tg((m->w[l] + 31) / 32, (m->w[l + 1] + 31) / 32);
    k_transpose_bf16<<<tg, tb, 0, m->stream>>>(m->Wb[l], m->WbT[l], m->w[l + 1], m->w[l]);
}

void transpose(mpm_mlp *m, const __nv_bfloat16 *in, __nv_bfloat16 *out, int rows, int cols)
{
    dim3 tb(32, 8), tg((cols + 31) / 32, (rows + 31) / 32);
    k_transpose_bf16<<<tg, tb, 0, m->stream>>>(in, out, rows, cols);
}

int forward(mpm_mlp *m, int B)
{
    for (int l = 0; l < m->L; ++l) {
        const int K = m->w[l], N = m->w[l + 1];
        // z = x W^T + b with the activation fused into the GEMM epilogue
        UmmaEpi epi;
        epi.bias = m->b[l];
        if (l + 1 < m->L) {
            epi.mode = m->hidden_act == MPM_ACT_RELU ? kEpiBiasRelu : kEpiBiasGelu;
            epi.xnext = m->X[l + 1];
        } else {
            epi.mode = m->out_act == MPM_OUT_LINEAR ? kEpiBiasLinear : kEpiBiasSigmoid;
            epi.y = m->Y;
            epi.lo = m->lo;
            epi.hi = m->hi;
        }
        cudaError_t e = umma_gemm_tma(B, N, K, m->X[l], K, m->Wb[l], K, m->Z[l], N, epi, m->status, m->stream);
        if (e != cudaSuccess) {
            m->err = std::string("gemm launch: ") + cudaGetErrorString(e);
            return MPM_ECUDA;
        }
    }
    return MPM_OK;
}

int check(mpm_mlp *m)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        m->err = cudaGetErrorString(e);
        return MPM_ECUDA;
    }
    return MPM_OK;
}

int sync_status(mpm_mlp *m)
{
    int32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, m->status, sizeof st, cudaMemcpyDeviceToHost, m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        m->err = cudaGetErrorString(e);
        return MPM_ECUDA;
    }
    if (st & kStatusTimeout) {
        m->err = "a bounded tensor-core wait ran out";
        return MPM_ETIMEOUT;
    }
    return MPM_OK;
}

int load_x(mpm_mlp *m, int B, const float *x, bool device)
{
    const int64_t n = (int64_t)B * m->w[0];
    const float *src = x;
    if (!device) {
        if (cudaMemcpyAsync(m->X0f, x, sizeof(float) * n, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
            return MPM_ECUDA;
        src = m->X0f;
    }
    k_f32_to_bf16<<<blocks_for(n), 256, 0, m->stream>>>(src, m->X[0], n);
    return MPM_OK;
}

// Back-propagation from dZ[L - 1] (already holding dL/dz of the output layer)
// and, with update, one Adam step.
int backward_update(mpm_mlp *m, int B, double lr, int update)
{
    const int L = m->L;
    for (int l = L - 1; l >= 0; --l) {
        const int Kin = m->w[l], N = m->w[l + 1];
        const int64_t nz = (int64_t)B * N;
        k_f32_to_bf16<<<blocks_for(nz), 256, 0, m->stream>>>(m->dZ[l], m->dZb[l], nz);
        transpose(m, m->dZb[l], m->dZbT[l], B, N);          // N x B
        transpose(m, m->X[l], m->XT[l], B, Kin);             // Kin x B
        // dW = dZ^T X : (N x B) (Kin x B)^T
        cudaError_t e = umma_gemm_tma(N, Kin, B, m->dZbT[l], B, m->XT[l], B, m->gW[l], Kin, UmmaEpi{}, m->status,
                                      m->stream);
        if (e != cudaSuccess) return MPM_ECUDA;
        k_col_sum<<<(N + 255) / 256, 256, 0, m->stream>>>(m->dZ[l], m->gb[l], B, N);
        if (l > 0) {
            // dA = dZ W : (B x N) (Kin x N)^T
            e = umma_gemm_tma(B, Kin, N, m->dZb[l], N, m->WbT[l], N, m->dA, Kin, UmmaEpi{}, m->status, m->stream);
            if (e != cudaSuccess) return MPM_ECUDA;
            k_act_back<<<blocks_for((int64_t)B * Kin), 256, 0, m->stream>>>(m->dA, m->Z[l - 1], m->dZ[l - 1],
                                                                           (int64_t)B * Kin,
                                                                           m->hidden_act == MPM_ACT_RELU);
        }
    }
    if (update) {
        m->step++;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
        for (int l = 0; l < L; ++l) {
            const int64_t nw = (int64_t)m->w[l + 1] * m->w[l], nb = m->w[l + 1];
            k_adam<<<blocks_for(nw), 256, 0, m->stream>>>(m->W[l], m->gW[l], m->mW[l], m->vW[l], nw, (float)lr, b1, b2,
                                                          1e-8f, c1, c2);
            k_adam<<<blocks_for(nb), 256, 0, m->stream>>>(m->b[l], m->gb[l], m->mb[l], m->vb[l], nb, (float)lr, b1, b2,
                                                          1e-8f, c1, c2);
            refresh_bf16(m, l);
        }
    }
    return MPM_OK;
}

// Queue one training step on the mean squared error (no synchronisation).
int train_queue(mpm_mlp *m, int B, const float *x, const float *target, double lr, int update, bool device)
{
    const int L = m->L;
    int rc = load_x(m, B, x, device);
    if (rc != MPM_OK) return rc;
    const int64_t nout = (int64_t)B * m->w[L];
    if (cudaMemcpyAsync(m->T, target, sizeof(float) * nout, device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        m->stream) != cudaSuccess)
        return MPM_ECUDA;
    rc = forward(m, B);
    if (rc != MPM_OK) return rc;
    cudaMemsetAsync(m->loss, 0, sizeof(double), m->stream);
    k_mse_out<<<blocks_for(nout), 256, 0, m->stream>>>(m->Y, m->T, m->Z[L - 1], m->dZ[L - 1], nout, m->lo, m->hi,
                                                      m->loss, m->out_act == MPM_OUT_LINEAR);
    rc = backward_update(m, B, lr, update);
    return rc != MPM_OK ? rc : check(m);
}

}  // namespace

extern "C" {

int mpm_gemm_bf16(int M, int N, int K, const void *A, int lda, const void *B, int ldb, float *C, int ldc,
                  int32_t *status_dev, void *cuda_stream)
{
    if (M <= 0 || N <= 0 || K <= 0 || !A || !B || !C || lda < K || ldb < K || ldc < N || (lda % 8) || (ldb % 8) ||
        !status_dev)
        return MPM_EINVAL;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) return MPM_EINVAL;
    cudaError_t e = umma_gemm_tma(M, N, K, (const __nv_bfloat16 *)A, lda, (const __nv_bfloat16 *)B, ldb, C, ldc, UmmaEpi{},
                              status_dev, (cudaStream_t)cuda_stream);
    return e == cudaSuccess ? MPM_OK : MPM_ECUDA;
}

int mpm_mlp_create(int n_layers, const int *widths, int max_batch, double out_lo, double out_hi, void *cuda_stream,
                   mpm_mlp **out)
{
    if (n_layers < 1 || n_layers > 8 || !widths || max_batch < 1 || max_batch > 65536 || !out || !(out_hi > out_lo))
        return MPM_EINVAL;
    for (int l = 0; l <= n_layers; ++l)
        if (widths[l] < 1 || widths[l] > 8192 || widths[l] % 8) return MPM_EINVAL;
    mpm_mlp *m = new mpm_mlp();
    m->L = n_layers;
    m->max_batch = (max_batch + 7) / 8 * 8;
    m->w.assign(widths, widths + n_layers + 1);
    m->lo = (float)out_lo;
    m->hi = (float)out_hi;
    if (cuda_stream) {
        m->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete m;
            return MPM_ECUDA;
        }
        m->own_stream = true;
    }
    const int L = n_layers, B = m->max_batch;
    int rc = MPM_OK;
    auto resize = [&](auto &v) { v.assign(L, nullptr); };
    resize(m->W); resize(m->b); resize(m->gW); resize(m->gb); resize(m->mW); resize(m->vW); resize(m->mb);
    resize(m->vb); resize(m->Wb); resize(m->WbT); resize(m->X); resize(m->XT); resize(m->Z); resize(m->dZ);
    resize(m->dZb); resize(m->dZbT);
    int maxw = 0;
    for (int l = 0; l <= L; ++l) maxw = std::max(maxw, widths[l]);
    for (int l = 0; l < L && rc == MPM_OK; ++l) {
        const size_t nw = (size_t)widths[l + 1] * widths[l], nb = widths[l + 1];
        rc = malloc_n(m, &m->W[l], nw);
        if (rc == MPM_OK) rc = malloc_n(m, &m->b[l], nb);
        if (rc == MPM_OK) rc = malloc_n(m, &m->gW[l], nw);
        if (rc == MPM_OK) rc = malloc_n(m, &m->gb[l], nb);
        if (rc == MPM_OK) rc = malloc_n(m, &m->mW[l], nw);
        if (rc == MPM_OK) rc = malloc_n(m, &m->vW[l], nw);
        if (rc == MPM_OK) rc = malloc_n(m, &m->mb[l], nb);
        if (rc == MPM_OK) rc = malloc_n(m, &m->vb[l], nb);
        if (rc == MPM_OK) rc = malloc_n(m, &m->Wb[l], nw);
        if (rc == MPM_OK) rc = malloc_n(m, &m->WbT[l], nw);
        if (rc == MPM_OK) rc = malloc_n(m, &m->X[l], (size_t)B * widths[l]);
        if (rc == MPM_OK) rc = malloc_n(m, &m->XT[l], (size_t)B * widths[l]);
        if (rc == MPM_OK) rc = malloc_n(m, &m->Z[l], (size_t)B * widths[l + 1]);
        if (rc == MPM_OK) rc = malloc_n(m, &m->dZ[l], (size_t)B * widths[l + 1]);
        if (rc == MPM_OK) rc = malloc_n(m, &m->dZb[l], (size_t)B * widths[l + 1]);
        if (rc == MPM_OK) rc = malloc_n(m, &m->dZbT[l], (size_t)B * widths[l + 1]);
    }
    if (rc == MPM_OK) rc = malloc_n(m, &m->Y, (size_t)B * widths[L]);
    if (rc == MPM_OK) rc = malloc_n(m, &m->T, (size_t)B * widths[L]);
    if (rc == MPM_OK) rc = malloc_n(m, &m->dA, (size_t)B * maxw);
    if (rc == MPM_OK) rc = malloc_n(m, &m->X0f, (size_t)B * widths[0]);
    if (rc == MPM_OK) rc = malloc_n(m, &m->loss, 1);
    if (rc == MPM_OK) rc = malloc_n(m, &m->status, 1);
    if (rc == MPM_OK && cudaMemsetAsync(m->status, 0, sizeof(int32_t), m->stream) != cudaSuccess) rc = MPM_ECUDA;
    if (rc != MPM_OK) {
        mpm_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return MPM_OK;
}

void mpm_mlp_destroy(mpm_mlp *m)
{
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (auto *vec : {&m->W, &m->b, &m->gW, &m->gb, &m->mW, &m->vW, &m->mb, &m->vb, &m->Z, &m->dZ})
        for (float *p : *vec)
            if (p) cudaFree(p);
    for (auto *vec : {&m->Wb, &m->WbT, &m->X, &m->XT, &m->dZb, &m->dZbT})
        for (__nv_bfloat16 *p : *vec)
            if (p) cudaFree(p);
    for (void *p : {(void *)m->Y, (void *)m->T, (void *)m->dA, (void *)m->X0f, (void *)m->loss, (void *)m->status})
        if (p) cudaFree(p);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

int64_t mpm_mlp_num_params(const mpm_mlp *m)
{
    if (!m) return MPM_EINVAL;
    int64_t n = 0;
    for (int l = 0; l < m->L; ++l) n += (int64_t)m->w[l + 1] * m->w[l] + m->w[l + 1];
    return n;
}

int mpm_mlp_set_params(mpm_mlp *m, const float *params)
{
    if (!m || !params) return MPM_EINVAL;
    const float *p = params;
    for (int l = 0; l < m->L; ++l) {
        const size_t nw = (size_t)m->w[l + 1] * m->w[l], nb = m->w[l + 1];
        if (cudaMemcpyAsync(m->W[l], p, sizeof(float) * nw, cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
            cudaMemcpyAsync(m->b[l], p + nw, sizeof(float) * nb, cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
            return MPM_ECUDA;
        cudaMemsetAsync(m->mW[l], 0, sizeof(float) * nw, m->stream);
        cudaMemsetAsync(m->vW[l], 0, sizeof(float) * nw, m->stream);
        cudaMemsetAsync(m->mb[l], 0, sizeof(float) * nb, m->stream);
        cudaMemsetAsync(m->vb[l], 0, sizeof(float) * nb, m->stream);
        refresh_bf16(m, l);
        p += nw + nb;
    }
    m->step = 0;
    int rc = check(m);
    return rc != MPM_OK ? rc : sync_status(m);
}

int mpm_mlp_get_params(mpm_mlp *m, float *params, int which)
{
    if (!m || !params || which < 0 || which > 1) return MPM_EINVAL;
    float *p = params;
    for (int l = 0; l < m->L; ++l) {
        const size_t nw = (size_t)m->w[l + 1] * m->w[l], nb = m->w[l + 1];
        const float *sw = which == 0 ? m->W[l] : m->gW[l];
        const float *sb = which == 0 ? m->b[l] : m->gb[l];
        if (cudaMemcpyAsync(p, sw, sizeof(float) * nw, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
            cudaMemcpyAsync(p + nw, sb, sizeof(float) * nb, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
            return MPM_ECUDA;
        p += nw + nb;
    }
    return sync_status(m);
}

int mpm_mlp_infer(mpm_mlp *m, int batch, const float *x, float *y, int device_ptrs)
{
    if (!m || !x || !y || batch < 1 || batch > m->max_batch) return MPM_EINVAL;
    int rc = load_x(m, batch, x, device_ptrs != 0);
    if (rc == MPM_OK) rc = forward(m, batch);
    if (rc == MPM_OK) rc = check(m);
    if (rc != MPM_OK) return rc;
    const size_t n = (size_t)batch * m->w[m->L];
    if (cudaMemcpyAsync(y, m->Y, sizeof(float) * n, device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        m->stream) != cudaSuccess)
        return MPM_ECUDA;
    return sync_status(m);
}

int mpm_mlp_train_step(mpm_mlp *m, int batch, const float *x, const float *target, double lr, int update,
                       double *loss_out, int device_ptrs)
{
    if (!m || !x || !target || batch < 8 || batch > m->max_batch || (batch % 8) || !(lr >= 0)) return MPM_EINVAL;
    int rc = train_queue(m, batch, x, target, lr, update, device_ptrs != 0);
    if (rc != MPM_OK) return rc;
    if (loss_out &&
        cudaMemcpyAsync(loss_out, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
        return MPM_ECUDA;
    return sync_status(m);
}

int mpm_mlp_train_step_async(mpm_mlp *m, int batch, const float *x_dev, const float *target_dev, double lr,
                             double *loss_dev)
{
    if (!m || !x_dev || !target_dev || batch < 8 || batch > m->max_batch || (batch % 8) || !(lr >= 0))
        return MPM_EINVAL;
    int rc = train_queue(m, batch, x_dev, target_dev, lr, 1, true);
    if (rc != MPM_OK) return rc;
    if (loss_dev &&
        cudaMemcpyAsync(loss_dev, m->loss, sizeof(double), cudaMemcpyDeviceToDevice, m->stream) != cudaSuccess)
        return MPM_ECUDA;
    return MPM_OK;
}

int mpm_mlp_backward(mpm_mlp *m, int batch, const float *x, const float *dy, double lr, int update, int device_ptrs)
{
    if (!m || !x || !dy || batch < 8 || batch > m->max_batch || (batch % 8) || !(lr >= 0)) return MPM_EINVAL;
    const int L = m->L;
    int rc = load_x(m, batch, x, device_ptrs != 0);
    if (rc == MPM_OK) rc = forward(m, batch);
    if (rc != MPM_OK) return rc;
    const int64_t nout = (int64_t)batch * m->w[L];
    if (cudaMemcpyAsync(m->T, dy, sizeof(float) * nout, device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        m->stream) != cudaSuccess)
        return MPM_ECUDA;
    k_out_back<<<blocks_for(nout), 256, 0, m->stream>>>(m->T, m->Z[L - 1], m->dZ[L - 1], nout, m->lo, m->hi,
                                                       m->out_act == MPM_OUT_LINEAR);
    rc = backward_update(m, batch, lr, update);
    if (rc == MPM_OK) rc = check(m);
    return rc != MPM_OK ? rc : sync_status(m);
}

int mpm_mlp_set_activations(mpm_mlp *m, int hidden, int output)
{
    if (!m || (hidden != MPM_ACT_GELU && hidden != MPM_ACT_RELU) ||
        (output != MPM_OUT_SIGMOID && output != MPM_OUT_LINEAR))
        return MPM_EINVAL;
    m->hidden_act = hidden;
    m->out_act = output;
    return MPM_OK;
}

int mpm_mlp_last_error(const mpm_mlp *m, char *buf, int len)
{
    if (!m || !buf || len <= 0) return MPM_EINVAL;
    std::snprintf(buf, (size_t)len, "%s", m->err.c_str());
    return MPM_OK;
}

}  // extern "C"
