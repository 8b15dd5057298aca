// The pivot-proposer network (not in the paper): a two-hidden-layer perceptron that scores
// candidate rows and columns of a Pi block, with its training kernels.
//
// Parameters are one flat FP32 vector for F inputs and H = 128 units per hidden layer:
//     W1 (H x F), b1 (H), W2 (H x H), b2 (H), W3 (H), b3 (1)
// Forward: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), z = W3 . h2 + b3 (one logit per sample).
// With fp16 weights every weight is rounded to FP16 before use (the inference form).
// Loss: mean over samples of w_s BCE(sigmoid(z_s), y_s), w_s = pos_weight for y_s = 1, else 1.
// Training kernels: the logit gradient, the input gradient of a layer (W^T g masked by the
// ReLU), weight gradients as tiled outer-product accumulations over the samples, bias
// gradients as column sums, and Adam (Kingma and Ba, 2015) with bias correction. Sums over
// samples go through FP32 atomics: gradients agree with a float64 reference to FP32 rounding.
#include <cuda_fp16.h>

#include "aci_internal.h"

namespace aci {

namespace {

constexpr int kH = kMlpHidden;
constexpr int kTileS = 16;  // samples per forward CTA

__device__ __forceinline__ float wcast(float w, int fp16) { return fp16 ? __half2float(__float2half_rn(w)) : w; }

// One CTA = kTileS samples, kH threads (thread j = hidden unit j). Saves the pre-activations
// a1, a2 (n x H) when they are given (training).
__global__ void __launch_bounds__(kH) mlp_forward_kernel(int n, int F, const float* __restrict__ X,
                                                         const float* __restrict__ P, int fp16, float* __restrict__ z,
                                                         float* __restrict__ a1s, float* __restrict__ a2s) {
    __shared__ float xs[kTileS][kMlpMaxInputs];
    __shared__ float h1[kTileS][kH];
    __shared__ float red[kTileS][kH / 32];
    const float* W1 = P;
    const float* b1 = W1 + kH * F;
    const float* W2 = b1 + kH;
    const float* b2 = W2 + kH * kH;
    const float* W3 = b2 + kH;
    const float* b3 = W3 + kH;
    const int j = threadIdx.x, s0 = blockIdx.x * kTileS;
    for (int e = j; e < kTileS * F; e += kH) {
        const int s = e / F, f = e % F;
        xs[s][f] = (s0 + s < n) ? X[(size_t)(s0 + s) * F + f] : 0.f;
    }
    __syncthreads();
    // layer 1
    float w1[kMlpMaxInputs];
    for (int f = 0; f < F; ++f) w1[f] = wcast(W1[j * F + f], fp16);
    const float bj1 = wcast(b1[j], fp16);
    for (int s = 0; s < kTileS; ++s) {
        float acc = bj1;
        for (int f = 0; f < F; ++f) acc = fmaf(w1[f], xs[s][f], acc);
        if (a1s && s0 + s < n) a1s[(size_t)(s0 + s) * kH + j] = acc;
        h1[s][j] = fmaxf(acc, 0.f);
    }
    __syncthreads();
    // layer 2: row j of W2 against every sample's h1
    float acc2[kTileS];
    const float bj2 = wcast(b2[j], fp16);
#pragma unroll
    for (int s = 0; s < kTileS; ++s) acc2[s] = bj2;
    for (int i = 0; i < kH; ++i) {
        const float w = wcast(W2[j * kH + i], fp16);
#pragma unroll
        for (int s = 0; s < kTileS; ++s) acc2[s] = fmaf(w, h1[s][i], acc2[s]);
    }
    const float w3 = wcast(W3[j], fp16);
    const int lane = j & 31, warp = j >> 5;
#pragma unroll
    for (int s = 0; s < kTileS; ++s) {
        if (a2s && s0 + s < n) a2s[(size_t)(s0 + s) * kH + j] = acc2[s];
        float t = w3 * fmaxf(acc2[s], 0.f);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (lane == 0) red[s][warp] = t;
    }
    __syncthreads();
    if (j < kTileS && s0 + j < n) {
        float t = wcast(b3[0], fp16);
        for (int w = 0; w < kH / 32; ++w) t += red[j][w];
        z[s0 + j] = t;
    }
}

// dz_s = w_s (sigmoid(z_s) - y_s) / n, and the mean loss (into *loss, FP64 atomics).
__global__ void mlp_dz_kernel(int n, const float* z, const float* y, float pos_weight, float* dz, double* loss) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (s < n) {
        const float zz = z[s], yy = y[s];
        const float w = yy > 0.5f ? pos_weight : 1.f;
        const float sig = 1.f / (1.f + __expf(-zz));
        dz[s] = w * (sig - yy) / (float)n;
        l = (double)w * (fmaxf(zz, 0.f) - zz * yy + log1pf(__expf(-fabsf(zz)))) / (double)n;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss, l);
}

// G_in[s][i] = (sum_j W[j][i] G_out[s][j]) * [a_in[s][i] > 0], W (Jd x Id) row-major; G_out (n x Jd).
// For the last layer Jd = 1 and G_out = dz (W3 is 1 x H).
__global__ void mlp_backprop_kernel(int n, int Id, int Jd, const float* W, const float* gout, const float* ain,
                                    float* gin) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * Id) return;
    const int s = (int)(e / Id), i = (int)(e % Id);
    float acc = 0.f;
    for (int j = 0; j < Jd; ++j) acc = fmaf(W[(size_t)j * Id + i], gout[(size_t)s * Jd + j], acc);
    gin[e] = ain[e] > 0.f ? acc : 0.f;
}

// C[p][q] += sum_s A[s][p] * act(B[s][q]) over a chunk of samples; act = relu when relu_b.
// Block 16 x 16 over a (p, q) tile, 64 samples per chunk staged in shared memory.
__global__ void mlp_outer_kernel(int n, int Pd, int Qd, const float* A, const float* B, int relu_b, float* C) {
    __shared__ float As[64][16];
    __shared__ float Bs[64][17];
    const int tp = threadIdx.y, tq = threadIdx.x;
    const int p = blockIdx.y * 16 + tp, q = blockIdx.x * 16 + tq;
    float acc = 0.f;
    for (int s0 = blockIdx.z * 64; s0 < n; s0 += gridDim.z * 64) {
        for (int e = tp * 16 + tq; e < 64 * 16; e += 256) {
            const int s = e / 16, c = e % 16;
            const int gs = s0 + s;
            As[s][c] = (gs < n && blockIdx.y * 16 + c < Pd) ? A[(size_t)gs * Pd + blockIdx.y * 16 + c] : 0.f;
            float bv = (gs < n && blockIdx.x * 16 + c < Qd) ? B[(size_t)gs * Qd + blockIdx.x * 16 + c] : 0.f;
            Bs[s][c] = relu_b ? fmaxf(bv, 0.f) : bv;
        }
        __syncthreads();
#pragma unroll 8
        for (int s = 0; s < 64; ++s) acc = fmaf(As[s][tp], Bs[s][tq], acc);
        __syncthreads();
    }
    if (p < Pd && q < Qd && acc != 0.f) atomicAdd(&C[(size_t)p * Qd + q], acc);
}

// out[p] += sum_s A[s][p]
__global__ void mlp_colsum_kernel(int n, int Pd, const float* A, float* out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Pd) return;
    float acc = 0.f;
    for (int s = blockIdx.y; s < n; s += gridDim.y) acc += A[(size_t)s * Pd + p];
    atomicAdd(&out[p], acc);
}

__global__ void mlp_adam_kernel(int count, float* p, const float* g, float* m, float* v, float lr, float b1,
                                float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

size_t mlp_param_count(int F) { return (size_t)kH * F + kH + (size_t)kH * kH + kH + kH + 1; }
size_t mlp_train_scratch(int n) { return (size_t)n * (4 * kH + 2); }

void launch_mlp_forward(int n, int F, const float* X, const float* P, int fp16, float* z, float* a1, float* a2,
                        cudaStream_t st) {
    if (n <= 0) return;
    mlp_forward_kernel<<<(n + kTileS - 1) / kTileS, kH, 0, st>>>(n, F, X, P, fp16, z, a1, a2);
}

void launch_mlp_grad(int n, int F, const float* X, const float* y, float pos_weight, const float* P, float* G,
                     double* loss, float* scratch, cudaStream_t st) {
    if (n <= 0) return;
    float* a1 = scratch;
    float* a2 = a1 + (size_t)n * kH;
    float* d2 = a2 + (size_t)n * kH;
    float* d1 = d2 + (size_t)n * kH;
    float* z = d1 + (size_t)n * kH;
    float* dz = z + n;
    const float* W2 = P + (size_t)kH * F + kH;
    const float* W3 = W2 + (size_t)kH * kH + kH;
    float* gW1 = G;
    float* gb1 = gW1 + (size_t)kH * F;
    float* gW2 = gb1 + kH;
    float* gb2 = gW2 + (size_t)kH * kH;
    float* gW3 = gb2 + kH;
    float* gb3 = gW3 + kH;
    cudaMemsetAsync(G, 0, sizeof(float) * mlp_param_count(F), st);
    cudaMemsetAsync(loss, 0, sizeof(double), st);
    launch_mlp_forward(n, F, X, P, 0, z, a1, a2, st);
    mlp_dz_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, z, y, pos_weight, dz, loss);
    const int chunks = std::min(64, std::max(1, n / 2048));
    // layer 3: dW3 = sum_s dz relu(a2) (a 1 x H outer product), db3 = sum dz, d2 = dz W3 [a2 > 0]
    mlp_outer_kernel<<<dim3((kH + 15) / 16, 1, chunks), dim3(16, 16), 0, st>>>(n, 1, kH, dz, a2, 1, gW3);
    mlp_colsum_kernel<<<dim3(1, std::min(n, 256)), 32, 0, st>>>(n, 1, dz, gb3);
    mlp_backprop_kernel<<<(unsigned)(((size_t)n * kH + 255) / 256), 256, 0, st>>>(n, kH, 1, W3, dz, a2, d2);
    // layer 2: dW2 = sum_s d2 (x) relu(a1), db2 = sum d2, d1 = W2^T d2 [a1 > 0]
    mlp_outer_kernel<<<dim3((kH + 15) / 16, (kH + 15) / 16, chunks), dim3(16, 16), 0, st>>>(n, kH, kH, d2, a1, 1, gW2);
    mlp_colsum_kernel<<<dim3((kH + 31) / 32, std::min(n, 256)), 32, 0, st>>>(n, kH, d2, gb2);
    mlp_backprop_kernel<<<(unsigned)(((size_t)n * kH + 255) / 256), 256, 0, st>>>(n, kH, kH, W2, d2, a1, d1);
    // layer 1: dW1 = sum_s d1 (x) x, db1 = sum d1
    mlp_outer_kernel<<<dim3((F + 15) / 16, (kH + 15) / 16, chunks), dim3(16, 16), 0, st>>>(n, kH, F, d1, X, 0, gW1);
    mlp_colsum_kernel<<<dim3((kH + 31) / 32, std::min(n, 256)), 32, 0, st>>>(n, kH, d1, gb1);
}

void launch_mlp_adam(int count, float* p, const float* g, float* m, float* v, int t, float lr, float b1, float b2,
                     float eps, cudaStream_t st) {
    if (count <= 0) return;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    mlp_adam_kernel<<<(count + 255) / 256, 256, 0, st>>>(count, p, g, m, v, lr, b1, b2, eps, c1, c2);
}

}  // namespace aci
