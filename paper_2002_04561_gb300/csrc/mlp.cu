// Band network: 64 k-mer diagonal features -> 128 -> 128 -> 2 (band centre,
// log half-width), ReLU after the hidden layers, bfloat16 weights with float32
// accumulation; forward, loss + backward (float32 gradients) and Adam with
// float32 master weights. The products are a few tens of thousands of
// multiply-adds per pair, negligible next to the pair's DP cells, so plain
// CUDA-core FMAs over shared-memory tiles are used.
//
// Loss per pair: Huber(c - c*, 8) / 8 + a(log w - log w*), a(r) = 4 r^2 for
// r < 0 (band too narrow) and r^2 otherwise; the batch loss is the mean.
#include <cuda_bf16.h>

#include "band.h"

namespace anyseq {

constexpr int TILE = 32;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_IN * MLP_H, OFF_W2 = OFF_B1 + MLP_H, OFF_B2 = OFF_W2 + MLP_H * MLP_H,
              OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_H * MLP_OUT;

__device__ __forceinline__ float bf(uint16_t w) { return __uint_as_float((uint32_t)w << 16); }

struct MlpSmem {
    uint16_t W1[MLP_IN * MLP_H];
    uint16_t W2[MLP_H * MLP_H];
    uint16_t W3[MLP_H * MLP_OUT];
    float b1[MLP_H], b2[MLP_H], b3[MLP_OUT];
    float X[TILE][MLP_IN];
    float H1[TILE][MLP_H];
    float H2[TILE][MLP_H];
    float G2[TILE][MLP_H];  // dL/dz2
    float GY[TILE][MLP_OUT];
};

__device__ void load_weights(MlpSmem &S, const MlpDev &P) {
    for (int k = threadIdx.x; k < MLP_IN * MLP_H; k += blockDim.x) S.W1[k] = P.w16[OFF_W1 + k];
    for (int k = threadIdx.x; k < MLP_H * MLP_H; k += blockDim.x) S.W2[k] = P.w16[OFF_W2 + k];
    for (int k = threadIdx.x; k < MLP_H * MLP_OUT; k += blockDim.x) S.W3[k] = P.w16[OFF_W3 + k];
    for (int k = threadIdx.x; k < MLP_H; k += blockDim.x) { S.b1[k] = P.master[OFF_B1 + k]; S.b2[k] = P.master[OFF_B2 + k]; }
    if (threadIdx.x < MLP_OUT) S.b3[threadIdx.x] = P.master[OFF_B3 + threadIdx.x];
}

// hidden layers of one tile (thread t = hidden unit t); rows beyond B are zero
__device__ void tile_forward(MlpSmem &S, const float *x, int64_t base, int64_t B) {
    const int t = threadIdx.x;
    for (int k = t; k < TILE * MLP_IN; k += blockDim.x) {
        int s = k / MLP_IN, c = k % MLP_IN;
        S.X[s][c] = (base + s < B) ? x[(base + s) * MLP_IN + c] : 0.0f;
    }
    __syncthreads();
    float acc[TILE];
#pragma unroll
    for (int s = 0; s < TILE; s++) acc[s] = S.b1[t];
    for (int k = 0; k < MLP_IN; k++) {
        const float w = bf(S.W1[k * MLP_H + t]);
#pragma unroll
        for (int s = 0; s < TILE; s++) acc[s] = fmaf(S.X[s][k], w, acc[s]);
    }
#pragma unroll
    for (int s = 0; s < TILE; s++) S.H1[s][t] = fmaxf(acc[s], 0.0f);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < TILE; s++) acc[s] = S.b2[t];
    for (int k = 0; k < MLP_H; k++) {
        const float w = bf(S.W2[k * MLP_H + t]);
#pragma unroll
        for (int s = 0; s < TILE; s++) acc[s] = fmaf(S.H1[s][k], w, acc[s]);
    }
#pragma unroll
    for (int s = 0; s < TILE; s++) S.H2[s][t] = fmaxf(acc[s], 0.0f);
    __syncthreads();
}

__device__ __forceinline__ float out_unit(const MlpSmem &S, int s, int o) {
    float y = S.b3[o];
    for (int k = 0; k < MLP_H; k++) y = fmaf(S.H2[s][k], bf(S.W3[k * MLP_OUT + o]), y);
    return y;
}

__global__ void __launch_bounds__(MLP_H) mlp_forward_kernel(MlpDev P, const float *x, int64_t B, float *y) {
    extern __shared__ __align__(16) uint8_t raw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(raw);
    load_weights(S, P);
    __syncthreads();
    for (int64_t base = (int64_t)blockIdx.x * TILE; base < B; base += (int64_t)gridDim.x * TILE) {
        tile_forward(S, x, base, B);
        if (threadIdx.x < TILE * MLP_OUT) {
            int s = threadIdx.x / MLP_OUT, o = threadIdx.x % MLP_OUT;
            if (base + s < B) y[(base + s) * MLP_OUT + o] = out_unit(S, s, o);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(MLP_H) mlp_grad_kernel(MlpDev P, const float *x, const float *target, int64_t B,
                                                         float *loss) {
    extern __shared__ __align__(16) uint8_t raw[];
    MlpSmem &S = *reinterpret_cast<MlpSmem *>(raw);
    load_weights(S, P);
    __syncthreads();
    const int t = threadIdx.x;
    const float invB = 1.0f / (float)B;
    for (int64_t base = (int64_t)blockIdx.x * TILE; base < B; base += (int64_t)gridDim.x * TILE) {
        tile_forward(S, x, base, B);
        // outputs, loss and dL/dy
        if (t < TILE) {
            const int64_t p = base + t;
            float g0 = 0.0f, g1 = 0.0f, l = 0.0f;
            if (p < B) {
                const float y0 = out_unit(S, t, 0), y1 = out_unit(S, t, 1);
                const float dc = y0 - target[p * 2], r = y1 - target[p * 2 + 1];
                const float adc = fabsf(dc);
                l = (adc <= 8.0f ? 0.5f * dc * dc : 8.0f * (adc - 4.0f)) / 8.0f;
                g0 = (adc <= 8.0f ? dc : copysignf(8.0f, dc)) / 8.0f;
                const float wgt = r < 0.0f ? 4.0f : 1.0f;
                l += wgt * r * r;
                g1 = 2.0f * wgt * r;
            }
            S.GY[t][0] = g0 * invB;
            S.GY[t][1] = g1 * invB;
            for (int off = 16; off; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
            if (t == 0) atomicAdd(loss, l);
        }
        __syncthreads();
        // layer 3 and dL/dz2 (thread t = hidden unit t)
        {
            float gw0 = 0.0f, gw1 = 0.0f;
            const float w30 = bf(S.W3[t * MLP_OUT]), w31 = bf(S.W3[t * MLP_OUT + 1]);
            for (int s = 0; s < TILE; s++) {
                gw0 = fmaf(S.H2[s][t], S.GY[s][0], gw0);
                gw1 = fmaf(S.H2[s][t], S.GY[s][1], gw1);
                const float gh = S.GY[s][0] * w30 + S.GY[s][1] * w31;
                S.G2[s][t] = S.H2[s][t] > 0.0f ? gh : 0.0f;
            }
            atomicAdd(&P.grad[OFF_W3 + t * MLP_OUT], gw0);
            atomicAdd(&P.grad[OFF_W3 + t * MLP_OUT + 1], gw1);
            if (t < MLP_OUT) {
                float gb = 0.0f;
                for (int s = 0; s < TILE; s++) gb += S.GY[s][t];
                atomicAdd(&P.grad[OFF_B3 + t], gb);
            }
        }
        __syncthreads();
        // layer 2: dW2 column t, db2, and dL/dz1 into X's place after use
        {
            float gb = 0.0f;
            for (int s = 0; s < TILE; s++) gb += S.G2[s][t];
            atomicAdd(&P.grad[OFF_B2 + t], gb);
            for (int k = 0; k < MLP_H; k++) {
                float acc = 0.0f;
                for (int s = 0; s < TILE; s++) acc = fmaf(S.H1[s][k], S.G2[s][t], acc);
                atomicAdd(&P.grad[OFF_W2 + k * MLP_H + t], acc);
            }
        }
        // dL/dz1 for unit k = t: sum over the layer-2 units
        float g1[TILE];
#pragma unroll
        for (int s = 0; s < TILE; s++) g1[s] = 0.0f;
        for (int u = 0; u < MLP_H; u++) {
            const float w = bf(S.W2[t * MLP_H + u]);
#pragma unroll
            for (int s = 0; s < TILE; s++) g1[s] = fmaf(S.G2[s][u], w, g1[s]);
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < TILE; s++) S.G2[s][t] = S.H1[s][t] > 0.0f ? g1[s] : 0.0f;  // reuse as dL/dz1
        __syncthreads();
        {
            float gb = 0.0f;
            for (int s = 0; s < TILE; s++) gb += S.G2[s][t];
            atomicAdd(&P.grad[OFF_B1 + t], gb);
            for (int k = 0; k < MLP_IN; k++) {
                float acc = 0.0f;
                for (int s = 0; s < TILE; s++) acc = fmaf(S.X[s][k], S.G2[s][t], acc);
                atomicAdd(&P.grad[OFF_W1 + k * MLP_H + t], acc);
            }
        }
        __syncthreads();
    }
}

__global__ void mlp_adam_kernel(MlpDev P, float lr, float c1, float c2) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= MLP_NPARAM) return;
    const float g = P.grad[k];
    const float m = 0.9f * P.m[k] + 0.1f * g;
    const float v = 0.999f * P.v[k] + 0.001f * g * g;
    P.m[k] = m;
    P.v[k] = v;
    const float w = P.master[k] - lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
    P.master[k] = w;
    P.w16[k] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
}

__global__ void mlp_round_kernel(MlpDev P) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < MLP_NPARAM) P.w16[k] = __bfloat16_as_ushort(__float2bfloat16_rn(P.master[k]));
}

static int mlp_grid(int64_t B) {
    int64_t g = (B + TILE - 1) / TILE;
    return (int)(g < 1 ? 1 : (g > 1216 ? 1216 : g));
}

cudaError_t launch_mlp_forward(const MlpDev &P, const float *x, int64_t B, float *y, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
    mlp_forward_kernel<<<mlp_grid(B), MLP_H, sizeof(MlpSmem), st>>>(P, x, B, y);
    return cudaGetLastError();
}

cudaError_t launch_mlp_grad(const MlpDev &P, const float *x, const float *target, int64_t B, float *loss,
                            cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(MlpSmem));
    mlp_grad_kernel<<<mlp_grid(B), MLP_H, sizeof(MlpSmem), st>>>(P, x, target, B, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(const MlpDev &P, int64_t step, float lr, cudaStream_t st) {
    const float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
    mlp_adam_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(P, lr, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_mlp_round(const MlpDev &P, cudaStream_t st) {
    mlp_round_kernel<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(P);
    return cudaGetLastError();
}

}  // namespace anyseq
