// Learned precision router: a 12 -> 64 -> 64 -> 1 MLP with BF16 weights and
// FP32 accumulation that predicts, for a shell quartet inside the band
// tau32 < Q_ab Q_cd Dmax <= K tau32, y = log10(max|T| Dmax / (Q_ab Q_cd Dmax)),
// i.e. how far the quartet's largest integral times density sits below its
// Schwarz bound. The quartet runs in FP32 iff log10(B / tau32) + y <= 0. The
// rigorous bound still caps every routed quartet at K tau32.
//
// This header is compiled twice: into the runtime-compiled integral kernels
// (routing decisions) and into the library's training kernels. Every
// floating-point step uses an explicitly rounded intrinsic so that the FP64
// and FP32 integral kernels, compiled separately, reach bit-identical
// decisions for the same quartet (a quartet must land in exactly one tier).
#pragma once

#define JK_RT_NIN 12
#define JK_RT_NINP 16   // inputs padded
#define JK_RT_NH 64

// Device-side weights (built on the host from the FP32 master copy).
struct JkRouterDev {
    float mu[JK_RT_NINP], isd[JK_RT_NINP];               // feature normalisation
    unsigned short W1[JK_RT_NINP * JK_RT_NH];            // bf16, [in][hidden]
    float b1[JK_RT_NH];
    unsigned short W2[JK_RT_NH * JK_RT_NH];              // bf16, [in][out]
    float b2[JK_RT_NH];
    unsigned short W3[JK_RT_NH];                         // bf16
    float b3;
    float margin;                                        // added to the prediction (safety)
    float pad[2];
};

// Per shell pair, for the features (host-computed at init).
struct JkPairFeat {
    float lpmin, lpmax;   // ln of the smallest / largest primitive exponent sum
    float rab;            // |A - B| (bohr)
    float lq;             // log10 Q_ab
    float pcx, pcy, pcz;  // centre of the most diffuse primitive pair
    float lsum;           // l_a + l_b
};

__device__ __forceinline__ float jk_bf16f(unsigned short w) { return __uint_as_float(((unsigned)w) << 16); }

// Features of quartet (ab|cd) with bound B and density factor dmax.
__device__ __forceinline__ void jk_router_features(const JkPairFeat &fa, const JkPairFeat &fc, double B,
                                                   double dmax, double tau, float x[JK_RT_NIN])
{
    const float dx = __fadd_rn(fa.pcx, -fc.pcx), dy = __fadd_rn(fa.pcy, -fc.pcy), dz = __fadd_rn(fa.pcz, -fc.pcz);
    const float r2 = __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
    x[0] = fa.lpmin;
    x[1] = fa.lpmax;
    x[2] = fc.lpmin;
    x[3] = fc.lpmax;
    x[4] = fa.rab;
    x[5] = fc.rab;
    x[6] = __fsqrt_rn(r2);
    x[7] = fa.lq;
    x[8] = fc.lq;
    // log10 in double, rounded once to float: identical in every kernel
    x[9] = (float)log10(dmax > 1e-300 ? dmax : 1e-300);
    x[10] = __fadd_rn(fa.lsum, fc.lsum);
    x[11] = (float)log10(B / tau);
}

// Prediction y (log10 units) for one feature vector.
__device__ __forceinline__ float jk_router_eval(const JkRouterDev *__restrict__ R, const float x[JK_RT_NIN])
{
    float xn[JK_RT_NIN];
#pragma unroll
    for (int i = 0; i < JK_RT_NIN; ++i) xn[i] = __fmul_rn(__fadd_rn(x[i], -__ldg(&R->mu[i])), __ldg(&R->isd[i]));
    float h1[JK_RT_NH];
#pragma unroll 4
    for (int o = 0; o < JK_RT_NH; ++o) {
        float acc = __ldg(&R->b1[o]);
#pragma unroll
        for (int i = 0; i < JK_RT_NIN; ++i) acc = __fmaf_rn(xn[i], jk_bf16f(__ldg(&R->W1[i * JK_RT_NH + o])), acc);
        h1[o] = fmaxf(acc, 0.0f);
    }
    float y = __ldg(&R->b3);
#pragma unroll 2
    for (int o = 0; o < JK_RT_NH; ++o) {
        float acc = __ldg(&R->b2[o]);
#pragma unroll
        for (int i = 0; i < JK_RT_NH; ++i) acc = __fmaf_rn(h1[i], jk_bf16f(__ldg(&R->W2[i * JK_RT_NH + o])), acc);
        y = __fmaf_rn(fmaxf(acc, 0.0f), jk_bf16f(__ldg(&R->W3[o])), y);
    }
    return __fadd_rn(y, __ldg(&R->margin));
}

// FP32 route decision for a band quartet.
__device__ __forceinline__ bool jk_router_to_fp32(const JkRouterDev *__restrict__ R, const JkPairFeat &fa,
                                                  const JkPairFeat &fc, double B, double dmax, double tau)
{
    float x[JK_RT_NIN];
    jk_router_features(fa, fc, B, dmax, tau, x);
    const float y = jk_router_eval(R, x);
    return __fadd_rn(x[11], y) <= 0.0f;
}
