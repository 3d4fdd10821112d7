// Learned warm start for BMPL: the per-atom proposal network's support
// features and its training.
//
// Gram row norms ||A^T a_j|| (one of the network's inputs) are estimated with
// a Rademacher sketch: for z_t = sum_j s_tj a_j (s_tj = +-1 from a hash),
// E[(z_t^T a_j)^2] = sum_k (a_k^T a_j)^2, averaged over T sketch vectors.
//
// Training (offline, not part of a solve): examples (features, label) come from
// the selection kernel's example mode on the first correlation C0 = A^T B, with
// labels j in supp(x*) from reference solutions.  One thread runs the forward
// and backward pass of one example; a CTA reduces the gradients of its examples
// (the 64 x 64 layer as a small matrix product in shared memory) and adds them
// to a global accumulator; an Adam step follows every minibatch.
#include "mpl_internal.cuh"

namespace mpl {

namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

// Z (T x n): z_t = sum_j s_tj a_j.  One thread per (t, k).
__global__ void k_sketch(const float* __restrict__ A32, int n, int m, int T, float* __restrict__ Z) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (k >= n || t >= T) return;
    float acc = 0.f;
    for (int j = 0; j < m; ++j) {
        const float s = (mix64(((uint64_t)t << 32) ^ (uint64_t)j) & 1ull) ? 1.f : -1.f;
        acc = fmaf(s, __ldg(A32 + (size_t)j * n + k), acc);
    }
    Z[(size_t)t * n + k] = acc;
}

// rn_j = sqrt(mean_t C[t][j]^2), C = Z A^T rows (T x m).
__global__ void k_rownorm(const float* __restrict__ C, int m, int T, float* __restrict__ rn) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    float s = 0.f;
    for (int t = 0; t < T; ++t) {
        const float v = C[(size_t)t * m + j];
        s = fmaf(v, v, s);
    }
    rn[j] = sqrtf(s / (float)T);
}

constexpr int TR_THREADS = 128;

struct TrainSmem {
    float w[PROP_NPARAM];
    float h1[TR_THREADS][PROP_H + 1];
    float d2[TR_THREADS][PROP_H + 1];
    float gsmall[P_W2 - P_W1 + PROP_H + PROP_H + 1];  // W1, b1 | b2 | w3, b3 partial sums
    float loss;
};

// Forward + backward for a minibatch slice.  ex: examples (f0, f1, f2, y); perm:
// example order; grad: accumulator (PROP_NPARAM, trainable part used); loss_acc: sum of losses.
__global__ void __launch_bounds__(TR_THREADS) k_train_fwd_bwd(const float* __restrict__ w, const float* __restrict__ ex,
                                                              const int* __restrict__ perm, int off, int count,
                                                              float inv_batch, float* __restrict__ grad,
                                                              float* __restrict__ loss_acc, int* __restrict__ n_acc) {
    extern __shared__ __align__(16) unsigned char raw[];
    TrainSmem& sh = *reinterpret_cast<TrainSmem*>(raw);
    const int tid = threadIdx.x;
    for (int t = tid; t < PROP_NPARAM; t += blockDim.x) sh.w[t] = w[t];
    const int nsmall = P_W2 - P_W1;  // W1 + b1
    for (int t = tid; t < nsmall + 2 * PROP_H + 1; t += blockDim.x) sh.gsmall[t] = 0.f;
    if (tid == 0) sh.loss = 0.f;
    __syncthreads();
    const int e = blockIdx.x * blockDim.x + tid;
    bool live = e < count;
    float f[3] = {0.f, 0.f, 0.f}, y = 0.f;
    if (live) {
        const float* x = ex + (size_t)perm[off + e] * 4;
        f[0] = x[0]; f[1] = x[1]; f[2] = x[2]; y = x[3];
        live = y >= 0.f;  // empty slots carry y = -1
    }
    const float* W = sh.w;
    float xin[3];
    for (int q = 0; q < 3; ++q) xin[q] = (f[q] - W[P_MEAN + q]) / W[P_STD + q];
    float h1[PROP_H];
#pragma unroll
    for (int o = 0; o < PROP_H; ++o)
        h1[o] = fmaxf(W[P_B1 + o] + W[P_W1 + o * 3] * xin[0] + W[P_W1 + o * 3 + 1] * xin[1] + W[P_W1 + o * 3 + 2] * xin[2], 0.f);
    float z = W[P_B3];
    float a2[PROP_H];
    for (int o = 0; o < PROP_H; ++o) {
        float a = W[P_B2 + o];
#pragma unroll
        for (int q = 0; q < PROP_H; ++q) a = fmaf(W[P_W2 + o * PROP_H + q], h1[q], a);
        a2[o] = a;
        z = fmaf(W[P_W3 + o], fmaxf(a, 0.f), z);
    }
    // binary cross-entropy with logits, stable form; dz = sigmoid(z) - y (mean over the batch)
    const float loss = live ? fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z))) : 0.f;
    const float dz = live ? (1.f / (1.f + expf(-z)) - y) * inv_batch : 0.f;
    // layer 3 and the pre-activation gradient of layer 2
    for (int o = 0; o < PROP_H; ++o) {
        const float h2 = fmaxf(a2[o], 0.f);
        atomicAdd(&sh.gsmall[nsmall + PROP_H + o], dz * h2);                 // w3
        const float d2 = a2[o] > 0.f ? dz * W[P_W3 + o] : 0.f;
        sh.d2[tid][o] = d2;
        atomicAdd(&sh.gsmall[nsmall + o], d2);                               // b2
    }
    atomicAdd(&sh.gsmall[nsmall + 2 * PROP_H], dz);                         // b3
    for (int q = 0; q < PROP_H; ++q) sh.h1[tid][q] = h1[q];
    atomicAdd(&sh.loss, loss);
    // layer 1: dh1 = W2^T d2 masked by ReLU
    for (int q = 0; q < PROP_H; ++q) {
        float a = 0.f;
        for (int o = 0; o < PROP_H; ++o) a = fmaf(W[P_W2 + o * PROP_H + q], sh.d2[tid][o], a);
        const float d1 = h1[q] > 0.f ? a : 0.f;
        atomicAdd(&sh.gsmall[q * 3 + 0], d1 * xin[0]);                       // W1
        atomicAdd(&sh.gsmall[q * 3 + 1], d1 * xin[1]);
        atomicAdd(&sh.gsmall[q * 3 + 2], d1 * xin[2]);
        atomicAdd(&sh.gsmall[PROP_H * 3 + q], d1);                           // b1
    }
    __syncthreads();
    // W2 gradient: sum over the CTA's examples of d2[e][o] * h1[e][q]
    for (int t = tid; t < PROP_H * PROP_H; t += blockDim.x) {
        const int o = t / PROP_H, q = t - o * PROP_H;
        float a = 0.f;
        for (int r = 0; r < TR_THREADS; ++r) a = fmaf(sh.d2[r][o], sh.h1[r][q], a);
        atomicAdd(&grad[P_W2 + t], a);
    }
    for (int t = tid; t < nsmall; t += blockDim.x) atomicAdd(&grad[P_W1 + t], sh.gsmall[t]);
    for (int t = tid; t < PROP_H; t += blockDim.x) {
        atomicAdd(&grad[P_B2 + t], sh.gsmall[nsmall + t]);
        atomicAdd(&grad[P_W3 + t], sh.gsmall[nsmall + PROP_H + t]);
    }
    if (tid == 0) {
        atomicAdd(&grad[P_B3], sh.gsmall[nsmall + 2 * PROP_H]);
        atomicAdd(loss_acc, sh.loss);
    }
    const int nlive = __syncthreads_count(live);
    if (tid == 0) atomicAdd(n_acc, nlive);
}

// Adam on the trainable parameters; clears the gradient.  step is 1-based.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ grad, float* __restrict__ m1, float* __restrict__ m2,
                       float lr, int step) {
    const int t = PROP_FIRST_TRAINABLE + blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= PROP_NPARAM) return;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float g = grad[t];
    const float a = b1 * m1[t] + (1.f - b1) * g;
    const float b = b2 * m2[t] + (1.f - b2) * g * g;
    m1[t] = a;
    m2[t] = b;
    const float ah = a / (1.f - powf(b1, (float)step)), bh = b / (1.f - powf(b2, (float)step));
    w[t] -= lr * ah / (sqrtf(bh) + eps);
    grad[t] = 0.f;
}

// BF16-rounded copy of the parameters for inference (normalisation constants stay FP32).
__global__ void k_round_bf16(const float* __restrict__ w, float* __restrict__ wb) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= PROP_NPARAM) return;
    wb[t] = t < PROP_FIRST_TRAINABLE ? w[t] : __bfloat162float(__float2bfloat16_rn(w[t]));
}

}  // namespace

cudaError_t launch_sketch_rownorm(const float* A32, int n, int m, int T, float* Z, cudaStream_t s, int64_t* nl) {
    dim3 grid((n + 127) / 128, T);
    k_sketch<<<grid, 128, 0, s>>>(A32, n, m, T, Z);
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_rownorm(const float* C, int m, int T, float* rn, cudaStream_t s, int64_t* nl) {
    k_rownorm<<<(m + 255) / 256, 256, 0, s>>>(C, m, T, rn);
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_train_step(const float* w, const float* ex, const int* perm, int off, int count, float inv_batch,
                              float* grad, float* loss_acc, int* n_acc, cudaStream_t s, int64_t* nl) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_train_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(TrainSmem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int blocks = (count + TR_THREADS - 1) / TR_THREADS;
    if (blocks <= 0) return cudaSuccess;
    k_train_fwd_bwd<<<blocks, TR_THREADS, sizeof(TrainSmem), s>>>(w, ex, perm, off, count, inv_batch, grad, loss_acc,
                                                                   n_acc);
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_adam(float* w, float* grad, float* m1, float* m2, float lr, int step, cudaStream_t s, int64_t* nl) {
    const int cnt = PROP_NPARAM - PROP_FIRST_TRAINABLE;
    k_adam<<<(cnt + 255) / 256, 256, 0, s>>>(w, grad, m1, m2, lr, step);
    ++*nl;
    return cudaGetLastError();
}

cudaError_t launch_round_bf16(const float* w, float* wb, cudaStream_t s, int64_t* nl) {
    k_round_bf16<<<(PROP_NPARAM + 255) / 256, 256, 0, s>>>(w, wb);
    ++*nl;
    return cudaGetLastError();
}

}  // namespace mpl
