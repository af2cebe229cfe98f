// Training kernels of the learned precision router (compiled by nvcc into the
// library). Parameters theta (FP32 master copy), flat:
//   W1[16][64] b1[64] W2[64][64] b2[64] W3[64] b3      (5,313 values)
// The forward pass rounds every weight and every layer input (normalised
// features, hidden activations) to BF16 (round to nearest even) and
// accumulates in FP32, as the tensor-core inference in the integral kernels
// does; the backward pass treats each rounding as the identity. The
// loss is the pinball (quantile) loss, which biases the prediction upwards so
// that a quartet is sent to FP32 only when its largest integral is confidently
// small.
#pragma once
#include "jk_router.cuh"

#define JK_RT_OFF_W1 0
#define JK_RT_OFF_B1 (JK_RT_NINP * JK_RT_NH)
#define JK_RT_OFF_W2 (JK_RT_OFF_B1 + JK_RT_NH)
#define JK_RT_OFF_B2 (JK_RT_OFF_W2 + JK_RT_NH * JK_RT_NH)
#define JK_RT_OFF_W3 (JK_RT_OFF_B2 + JK_RT_NH)
#define JK_RT_OFF_B3 (JK_RT_OFF_W3 + JK_RT_NH)
#define JK_RT_NPARAM (JK_RT_OFF_B3 + 1)

__host__ __device__ inline unsigned short jk_f2bf(float f)
{
    unsigned u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return (unsigned short)(u >> 16);   // inf / nan
    u += 0x7fffu + ((u >> 16) & 1u);                                          // nearest even
    return (unsigned short)(u >> 16);
}
__host__ __device__ inline float jk_bf2f(unsigned short b)
{
    unsigned u = ((unsigned)b) << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// splitmix64: counter-based sample picker
__device__ __forceinline__ unsigned long long jk_mix64(unsigned long long z)
{
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// One mini-batch: forward, pinball loss, backward; gradients summed per CTA
// in shared memory and added to `grad` once per CTA. Sample t of the batch is
// row idx[t] if idx != nullptr, else a hashed row of X.
__global__ void jk_mlp_grad_kernel(const float *__restrict__ theta, const float *__restrict__ mu,
                                   const float *__restrict__ isd, const float *__restrict__ X,
                                   const float *__restrict__ y, long long n, const long long *__restrict__ idx,
                                   int batch, unsigned long long seed, float q, float *__restrict__ grad,
                                   double *__restrict__ loss)
{
    extern __shared__ float sm[];
    float *sw = sm;                       // BF16-rounded weights, as floats
    float *sg = sm + JK_RT_NPARAM;        // gradient accumulator
    for (int i = threadIdx.x; i < JK_RT_NPARAM; i += blockDim.x) {
        const bool is_w = (i < JK_RT_OFF_B1) || (i >= JK_RT_OFF_W2 && i < JK_RT_OFF_B2) ||
                          (i >= JK_RT_OFF_W3 && i < JK_RT_OFF_B3);
        sw[i] = is_w ? jk_bf2f(jk_f2bf(theta[i])) : theta[i];
        sg[i] = 0.0f;
    }
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double lsum = 0.0;
    if (t < batch) {
        long long row = idx ? idx[t] : (long long)(jk_mix64(seed * 0x100000001b3ull + (unsigned long long)t) % (unsigned long long)n);
        float xn[JK_RT_NINP];
        for (int i = 0; i < JK_RT_NINP; ++i) xn[i] = 0.0f;
        for (int i = 0; i < JK_RT_NIN; ++i)
            xn[i] = jk_bf2f(jk_f2bf(__fmul_rn(__fadd_rn(X[row * JK_RT_NIN + i], -mu[i]), isd[i])));
        float a1[JK_RT_NH], h1[JK_RT_NH];
        for (int o = 0; o < JK_RT_NH; ++o) {
            float acc = sw[JK_RT_OFF_B1 + o];
            for (int i = 0; i < JK_RT_NIN; ++i) acc = fmaf(xn[i], sw[JK_RT_OFF_W1 + i * JK_RT_NH + o], acc);
            a1[o] = acc;
            h1[o] = jk_bf2f(jk_f2bf(fmaxf(acc, 0.0f)));
        }
        float a2[JK_RT_NH];
        float out = sw[JK_RT_OFF_B3];
        for (int o = 0; o < JK_RT_NH; ++o) {
            float acc = sw[JK_RT_OFF_B2 + o];
            for (int i = 0; i < JK_RT_NH; ++i) acc = fmaf(h1[i], sw[JK_RT_OFF_W2 + i * JK_RT_NH + o], acc);
            a2[o] = acc;
            out = fmaf(jk_bf2f(jk_f2bf(fmaxf(acc, 0.0f))), sw[JK_RT_OFF_W3 + o], out);
        }
        const float u = y[row] - out;                 // pinball: u (q - [u < 0])
        lsum = (double)(u >= 0.0f ? q * u : (q - 1.0f) * u);
        const float g = (u < 0.0f ? 1.0f : 0.0f) - q;  // d loss / d out
        const float gs = g / (float)batch;
        atomicAdd(&sg[JK_RT_OFF_B3], gs);
        float dh1[JK_RT_NH];
        for (int i = 0; i < JK_RT_NH; ++i) dh1[i] = 0.0f;
        for (int o = 0; o < JK_RT_NH; ++o) {
            atomicAdd(&sg[JK_RT_OFF_W3 + o], gs * jk_bf2f(jk_f2bf(fmaxf(a2[o], 0.0f))));
            if (a2[o] > 0.0f) {
                const float d2 = gs * sw[JK_RT_OFF_W3 + o];
                atomicAdd(&sg[JK_RT_OFF_B2 + o], d2);
                for (int i = 0; i < JK_RT_NH; ++i) {
                    if (h1[i] != 0.0f) atomicAdd(&sg[JK_RT_OFF_W2 + i * JK_RT_NH + o], h1[i] * d2);
                    dh1[i] = fmaf(sw[JK_RT_OFF_W2 + i * JK_RT_NH + o], d2, dh1[i]);
                }
            }
        }
        for (int i = 0; i < JK_RT_NH; ++i) {
            if (a1[i] > 0.0f) {
                atomicAdd(&sg[JK_RT_OFF_B1 + i], dh1[i]);
                for (int k = 0; k < JK_RT_NIN; ++k)
                    if (xn[k] != 0.0f) atomicAdd(&sg[JK_RT_OFF_W1 + k * JK_RT_NH + i], xn[k] * dh1[i]);
            }
        }
    }
    // loss: warp sum, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0 && lsum != 0.0) atomicAdd(loss, lsum / batch);
    __syncthreads();
    for (int i = threadIdx.x; i < JK_RT_NPARAM; i += blockDim.x)
        if (sg[i] != 0.0f) atomicAdd(&grad[i], sg[i]);
}

__global__ void jk_adam_kernel(float *__restrict__ theta, const float *__restrict__ grad, float *__restrict__ m1,
                               float *__restrict__ m2, int step, float lr, float b1, float b2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= JK_RT_NPARAM) return;
    const float g = grad[i];
    const float a = b1 * m1[i] + (1.0f - b1) * g;
    const float v = b2 * m2[i] + (1.0f - b2) * g * g;
    m1[i] = a;
    m2[i] = v;
    const float ah = a / (1.0f - powf(b1, (float)step));
    const float vh = v / (1.0f - powf(b2, (float)step));
    theta[i] -= lr * ah / (sqrtf(vh) + eps);
}

// Inference over a batch of feature rows with the device weights (the same
// warp-level tensor-core function the integral kernels call). Blocks of 128
// threads; rows past n are evaluated on zero features and not stored.
__global__ void __launch_bounds__(128) jk_mlp_forward_kernel(const JkRouterDev *__restrict__ R,
                                                             const float *__restrict__ X, long long n,
                                                             float *__restrict__ out)
{
    __shared__ __align__(16) unsigned short s_rsm[4 * 32 * JK_RT_NINP];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float x[JK_RT_NIN];
    for (int i = 0; i < JK_RT_NIN; ++i) x[i] = t < n ? X[t * JK_RT_NIN + i] : 0.0f;
    const float y = jk_router_warp(R, x, s_rsm + (threadIdx.x >> 5) * 32 * JK_RT_NINP);
    if (t < n) out[t] = y;
}
