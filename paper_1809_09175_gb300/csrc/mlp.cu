// mlp.cu -- the learned schedule selector's network (not in the paper): a
// three-layer perceptron  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
// y = W3 h2 + b3  mapping per-mode features to predicted log run times of the
// candidate schedules.  Hand-written kernels for the forward pass, the masked
// mean-squared-error gradient (backward pass), Adam updates, and a fused
// one-CTA inference kernel used when a schedule is chosen.
//
// Parameters are packed: W1 (H1 x F), b1 (H1), W2 (H2 x H1), b2 (H2),
// W3 (K x H2), b3 (K); weight matrices row-major (out x in); samples are rows.
#include <cmath>
#include <vector>

#include "internal.h"

namespace spt {
namespace {

struct Layout {
    int64_t W1, b1, W2, b2, W3, b3, total;
};

Layout layout(int F, int H1, int H2, int K) {
    Layout L;
    L.W1 = 0;
    L.b1 = L.W1 + (int64_t)H1 * F;
    L.W2 = L.b1 + H1;
    L.b2 = L.W2 + (int64_t)H2 * H1;
    L.W3 = L.b2 + H2;
    L.b3 = L.W3 + (int64_t)K * H2;
    L.total = L.b3 + K;
    return L;
}

__global__ void dense_fwd_kernel(int B, int In, int Out, const float *X, const float *W,
                                 const float *bias, float *Y, int relu) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * Out) return;
    const int s = (int)(e / Out), o = (int)(e % Out);
    float acc = bias[o];
    for (int i = 0; i < In; ++i) acc = fmaf(W[(int64_t)o * In + i], X[(int64_t)s * In + i], acc);
    Y[e] = (relu && acc < 0.f) ? 0.f : acc;
}

__global__ void mask_sum_kernel(int64_t n, const float *M, float *msum, float *loss) {
    __shared__ float red[32];
    float a = 0.f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += M[i];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *msum = t > 0.f ? t : 1.f;
        *loss = 0.f;
    }
}

__global__ void out_grad_kernel(int64_t n, const float *Y, const float *T, const float *M,
                                const float *msum, float *gY, float *loss) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float l = 0.f;
    if (i < n) {
        const float e = Y[i] - T[i];
        gY[i] = 2.f * M[i] * e / *msum;
        l = M[i] * e * e / *msum;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l);
}

// dW[o][i] = sum_s G[s][o] X[s][i]  (i < In);  db[o] = sum_s G[s][o]  (i == In)
__global__ void dense_bwd_w_kernel(int B, int In, int Out, const float *G, const float *X, float *dW,
                                   float *db) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)Out * (In + 1)) return;
    const int o = (int)(e / (In + 1)), i = (int)(e % (In + 1));
    float acc = 0.f;
    if (i < In) {
        for (int s = 0; s < B; ++s) acc = fmaf(G[(int64_t)s * Out + o], X[(int64_t)s * In + i], acc);
        dW[(int64_t)o * In + i] = acc;
    } else {
        for (int s = 0; s < B; ++s) acc += G[(int64_t)s * Out + o];
        db[o] = acc;
    }
}

// gX[s][i] = relu'(Xact[s][i]) * sum_o W[o][i] G[s][o]
__global__ void dense_bwd_x_kernel(int B, int In, int Out, const float *G, const float *W,
                                   const float *Xact, float *gX) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)B * In) return;
    const int s = (int)(e / In), i = (int)(e % In);
    float acc = 0.f;
    for (int o = 0; o < Out; ++o) acc = fmaf(W[(int64_t)o * In + i], G[(int64_t)s * Out + o], acc);
    gX[e] = Xact[e] > 0.f ? acc : 0.f;
}

__global__ void adam_kernel(int64_t n, float *p, const float *g, float *m, float *v, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// One CTA evaluates the whole network for B samples (B small), layer by
// layer in shared memory.
__global__ void mlp_infer_kernel(int B, int F, int H1, int H2, int K, const float *X,
                                 const float *params, int64_t oW1, int64_t ob1, int64_t oW2,
                                 int64_t ob2, int64_t oW3, int64_t ob3, float *Y) {
    extern __shared__ float sm[];
    float *x = sm, *h1 = x + F, *h2 = h1 + H1;
    for (int s = 0; s < B; ++s) {
        for (int i = threadIdx.x; i < F; i += blockDim.x) x[i] = X[(int64_t)s * F + i];
        __syncthreads();
        for (int o = threadIdx.x; o < H1; o += blockDim.x) {
            float a = params[ob1 + o];
            for (int i = 0; i < F; ++i) a = fmaf(params[oW1 + (int64_t)o * F + i], x[i], a);
            h1[o] = a > 0.f ? a : 0.f;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < H2; o += blockDim.x) {
            float a = params[ob2 + o];
            for (int i = 0; i < H1; ++i) a = fmaf(params[oW2 + (int64_t)o * H1 + i], h1[i], a);
            h2[o] = a > 0.f ? a : 0.f;
        }
        __syncthreads();
        for (int o = threadIdx.x; o < K; o += blockDim.x) {
            float a = params[ob3 + o];
            for (int i = 0; i < H2; ++i) a = fmaf(params[oW3 + (int64_t)o * H2 + i], h2[i], a);
            Y[(int64_t)s * K + o] = a;
        }
        __syncthreads();
    }
}

inline int blocks_for(int64_t n) { return (int)std::max<int64_t>(1, (n + 255) / 256); }

spt_status forward_layers(int B, int F, int H1, int H2, int K, const float *X, const float *params,
                          float *h1, float *h2, float *Y, cudaStream_t st) {
    const Layout L = layout(F, H1, H2, K);
    dense_fwd_kernel<<<blocks_for((int64_t)B * H1), 256, 0, st>>>(B, F, H1, X, params + L.W1, params + L.b1, h1, 1);
    dense_fwd_kernel<<<blocks_for((int64_t)B * H2), 256, 0, st>>>(B, H1, H2, h1, params + L.W2, params + L.b2, h2, 1);
    dense_fwd_kernel<<<blocks_for((int64_t)B * K), 256, 0, st>>>(B, H2, K, h2, params + L.W3, params + L.b3, Y, 0);
    SPT_LAUNCH_CHECK("dense_fwd_kernel");
    return SPT_OK;
}

bool dims_ok(int B, int F, int H1, int H2, int K) {
    return B >= 1 && F >= 1 && H1 >= 1 && H2 >= 1 && K >= 1 && F <= 4096 && H1 <= 4096 &&
           H2 <= 4096 && K <= 4096;
}

}  // namespace
}  // namespace spt

using namespace spt;

extern "C" {

int64_t mlp_param_count(int F, int H1, int H2, int K) { return layout(F, H1, H2, K).total; }

int64_t mlp_workspace_floats(int B, int F, int H1, int H2, int K) {
    (void)F;
    return 2 * (int64_t)B * (H1 + H2 + K) + 64;
}

spt_status mlp_forward(int B, int F, int H1, int H2, int K, const float *X, const float *params,
                       float *Y, float *work, void *stream) {
    if (!dims_ok(B, F, H1, H2, K)) return fail(SPT_EINVAL, "mlp_forward: bad sizes");
    if (!X || !params || !Y || !work) return fail(SPT_EINVAL, "mlp_forward: NULL argument");
    float *h1 = work, *h2 = h1 + (int64_t)B * H1;
    return forward_layers(B, F, H1, H2, K, X, params, h1, h2, Y, (cudaStream_t)stream);
}

spt_status mlp_loss_grad(int B, int F, int H1, int H2, int K, const float *X, const float *params,
                         const float *T, const float *M, float *grads, float *loss, float *work,
                         void *stream) {
    if (!dims_ok(B, F, H1, H2, K)) return fail(SPT_EINVAL, "mlp_loss_grad: bad sizes");
    if (!X || !params || !T || !M || !grads || !loss || !work)
        return fail(SPT_EINVAL, "mlp_loss_grad: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    const Layout L = layout(F, H1, H2, K);
    float *h1 = work, *h2 = h1 + (int64_t)B * H1, *Y = h2 + (int64_t)B * H2;
    float *gY = Y + (int64_t)B * K, *g2 = gY + (int64_t)B * K, *g1 = g2 + (int64_t)B * H2;
    float *msum = g1 + (int64_t)B * H1;
    spt_status s = forward_layers(B, F, H1, H2, K, X, params, h1, h2, Y, st);
    if (s) return s;
    const int64_t nY = (int64_t)B * K;
    mask_sum_kernel<<<1, 1024, 0, st>>>(nY, M, msum, loss);
    out_grad_kernel<<<blocks_for(nY), 256, 0, st>>>(nY, Y, T, M, msum, gY, loss);
    dense_bwd_w_kernel<<<blocks_for((int64_t)K * (H2 + 1)), 256, 0, st>>>(B, H2, K, gY, h2, grads + L.W3, grads + L.b3);
    dense_bwd_x_kernel<<<blocks_for((int64_t)B * H2), 256, 0, st>>>(B, H2, K, gY, params + L.W3, h2, g2);
    dense_bwd_w_kernel<<<blocks_for((int64_t)H2 * (H1 + 1)), 256, 0, st>>>(B, H1, H2, g2, h1, grads + L.W2, grads + L.b2);
    dense_bwd_x_kernel<<<blocks_for((int64_t)B * H1), 256, 0, st>>>(B, H1, H2, g2, params + L.W2, h1, g1);
    dense_bwd_w_kernel<<<blocks_for((int64_t)H1 * (F + 1)), 256, 0, st>>>(B, F, H1, g1, X, grads + L.W1, grads + L.b1);
    SPT_LAUNCH_CHECK("mlp backward kernels");
    return SPT_OK;
}

spt_status mlp_adam(int64_t n, float *params, const float *grads, float *m, float *v, float lr,
                    float beta1, float beta2, float eps, int step, void *stream) {
    if (n < 1 || !params || !grads || !m || !v || step < 1) return fail(SPT_EINVAL, "mlp_adam: bad argument");
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(n, params, grads, m, v, lr, beta1,
                                                                 beta2, eps, c1, c2);
    SPT_LAUNCH_CHECK("adam_kernel");
    return SPT_OK;
}

spt_status mlp_infer(int B, int F, int H1, int H2, int K, const float *X, const float *params,
                     float *Y, void *stream) {
    if (!dims_ok(B, F, H1, H2, K)) return fail(SPT_EINVAL, "mlp_infer: bad sizes");
    if (!X || !params || !Y) return fail(SPT_EINVAL, "mlp_infer: NULL argument");
    const Layout L = layout(F, H1, H2, K);
    const size_t smem = sizeof(float) * (F + H1 + H2);
    if (smem > 48 * 1024) return fail(SPT_EUNSUPPORTED, "mlp_infer: layers too wide");
    mlp_infer_kernel<<<1, 256, smem, (cudaStream_t)stream>>>(B, F, H1, H2, K, X, params, L.W1, L.b1,
                                                             L.W2, L.b2, L.W3, L.b3, Y);
    SPT_LAUNCH_CHECK("mlp_infer_kernel");
    return SPT_OK;
}

spt_status mttkrp_select(spt_tensor t, int mode, spt_dtype fdt, int rank, const spt_selector *sel,
                         spt_schedule *out, float *pred, void *stream) {
    if (!t || !sel || !out || !sel->params) return fail(SPT_EINVAL, "mttkrp_select: NULL argument");
    if (sel->F != SPT_NUM_FEATURES || sel->K != SPT_NUM_CANDIDATES)
        return fail(SPT_EINVAL, "mttkrp_select: network must map SPT_NUM_FEATURES to SPT_NUM_CANDIDATES");
    float f[SPT_NUM_FEATURES];
    spt_status s = tensor_mode_features(t, mode, rank, fdt, f);
    if (s) return s;
    for (int i = 0; i < SPT_NUM_FEATURES; ++i) {
        const float mu = sel->mean ? sel->mean[i] : 0.f;
        const float sd = sel->std ? sel->std[i] : 1.f;
        f[i] = (f[i] - mu) / (sd > 0.f ? sd : 1.f);
    }
    cudaStream_t st = (cudaStream_t)stream;
    float *dx = nullptr;
    s = dmalloc((void **)&dx, sizeof(float) * (SPT_NUM_FEATURES + SPT_NUM_CANDIDATES), st);
    if (s) return s;
    float *dy = dx + SPT_NUM_FEATURES;
    float y[SPT_NUM_CANDIDATES];
    cudaError_t e = cudaMemcpyAsync(dx, f, sizeof(f), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        s = mlp_infer(1, sel->F, sel->H1, sel->H2, sel->K, dx, sel->params, dy, stream);
        if (!s) e = cudaMemcpyAsync(y, dy, sizeof(y), cudaMemcpyDeviceToHost, st);
        if (!s && e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    dfree(dx, st);
    if (s) return s;
    if (e != cudaSuccess) return cuda_fail(e, "mttkrp_select");
    spt_schedule cand[SPT_NUM_CANDIDATES];
    int valid[SPT_NUM_CANDIDATES];
    for (int q = 0; q < SPT_NUM_CANDIDATES; ++q) {
        cand[q] = candidate(q, rank);
        valid[q] = candidate_valid(t, mode, rank, fdt, cand[q], q) ? 1 : 0;
    }
    int bq = -1;
    for (int q = 0; q < SPT_NUM_CANDIDATES; ++q)
        if (valid[q] && (bq < 0 || y[q] < y[bq])) bq = q;
    if (pred)
        for (int q = 0; q < SPT_NUM_CANDIDATES; ++q) pred[q] = y[q];
    if (sel->anchor_margin >= 0.f && (bq < 0 || y[bq] >= -sel->anchor_margin)) {
        // outputs are relative to the library's own choice: keep it unless a
        // candidate is predicted to beat it by more than the margin
        *out = default_schedule(t, mode, fdt, rank);
        return SPT_OK;
    }
    if (bq < 0) return fail(SPT_EUNSUPPORTED, "mttkrp_select: no valid candidate");
    *out = cand[bq];
    return SPT_OK;
}

}  // extern "C"
