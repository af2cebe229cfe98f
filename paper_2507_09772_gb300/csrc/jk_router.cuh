// Learned precision router: a 12 -> 64 -> 64 -> 1 MLP with BF16 weights and
// FP32 accumulation that predicts, for a shell quartet inside the band
// tau32 < Q_ab Q_cd Dmax <= K tau32, y = log10(max|T| / (Q_ab Q_cd)), i.e.
// how far the quartet's largest integral sits below its Schwarz bound. The
// quartet runs in FP32 iff log10(B / tau32) + y + margin <= 0. The rigorous
// bound still caps every routed quartet at K tau32.
//
// Inference runs on the tensor cores, one warp at a time: the 32 candidates
// a screening warp holds are the rows of mma.sync.m16n8k16 (BF16 inputs,
// FP32 accumulation), 88 MMAs per warp for the three layers. The inputs of
// each layer (normalised features, hidden activations) are rounded to BF16;
// the training kernels and the CPU reference round the same way.
//
// This header is compiled into the runtime-compiled integral kernels (the
// FP64 tier of routed builds runs it) and into the library's training
// kernels. Every step is either an MMA (fixed accumulation order) or an
// explicitly rounded intrinsic, so a quartet's decision does not depend on
// the kernel or the launch that evaluates it.
#pragma once

#define JK_RT_NIN 12
#define JK_RT_NINP 16   // inputs padded
#define JK_RT_NH 64

// Device-side weights, built on the host from the FP32 master copy. The
// weight matrices are stored in the B-fragment order of mma.m16n8k16
// (per k-step, n-tile, lane: two 32-bit registers of two BF16 values each).
struct JkRouterDev {
    float mu[JK_RT_NINP], isd[JK_RT_NINP];   // feature normalisation
    float b1[JK_RT_NH], b2[JK_RT_NH];
    float b3, margin, pad[2];
    unsigned W1p[1 * 8 * 32 * 2];            // 16 x 64
    unsigned W2p[4 * 8 * 32 * 2];            // 64 x 64
    unsigned W3p[4 * 1 * 32 * 2];            // 64 x 8 (column 0 used)
};

// Per shell pair, for the features (host-computed at init).
struct alignas(16) JkPairFeat {
    float lpmin, lpmax;   // ln of the smallest / largest primitive exponent sum
    float rab;            // |A - B| (bohr)
    float lq;             // log10 Q_ab
    float pcx, pcy, pcz;  // centre of the most diffuse primitive pair
    float lsum;           // l_a + l_b
};

// float -> bf16 bits, round to nearest even (integer arithmetic only)
__device__ __forceinline__ unsigned jk_bf16_bits(float f)
{
    unsigned u = __float_as_uint(f);
    if ((u & 0x7f800000u) == 0x7f800000u) return u >> 16;
    return (u + 0x7fffu + ((u >> 16) & 1u)) >> 16;
}
__device__ __forceinline__ unsigned jk_pack_bf16(float lo, float hi)
{
    return jk_bf16_bits(lo) | (jk_bf16_bits(hi) << 16);
}

__device__ __forceinline__ void jk_mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Features of quartet (ab|cd) with bound B and density factor dmax.
__device__ __forceinline__ void jk_router_features(const JkPairFeat &fa, const JkPairFeat &fc, float B,
                                                   float dmax, float tau, float x[JK_RT_NIN])
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
    // FP32 logarithms (the FP64 ones cost dozens of FP64-pipe instructions
    // per lane); the same code in every kernel gives the same bits
    x[9] = log10f(fmaxf(dmax, 1e-30f));
    x[10] = __fadd_rn(fa.lsum, fc.lsum);
    x[11] = log10f(__fdiv_rn(B, tau));
}

// Prediction (margin included) for the candidate this lane holds; every lane
// of the warp must call it (warp-synchronous). sm: 32 x 16 BF16 scratch of
// this warp in shared memory.
__device__ __forceinline__ float jk_router_warp(const JkRouterDev *__restrict__ R, const float x[JK_RT_NIN],
                                                unsigned short *sm)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    // normalised features of this lane's candidate -> BF16 row `lane`
#pragma unroll
    for (int i = 0; i < JK_RT_NINP; ++i) {
        const float v = i < JK_RT_NIN ? __fmul_rn(__fadd_rn(x[i], -__ldg(&R->mu[i])), __ldg(&R->isd[i])) : 0.0f;
        sm[lane * JK_RT_NINP + i] = (unsigned short)jk_bf16_bits(v);
    }
    __syncwarp();
    const unsigned *smw = reinterpret_cast<const unsigned *>(sm);
    const uint2 *W1 = reinterpret_cast<const uint2 *>(R->W1p);
    const uint2 *W2 = reinterpret_cast<const uint2 *>(R->W2p);
    const uint2 *W3 = reinterpret_cast<const uint2 *>(R->W3p);
    // Each weight fragment is loaded once and applied to both 16-row tiles
    // at once; layer 2 is computed 16 output columns at a time and folded
    // straight into layer 3, so only the first hidden layer stays live.
    unsigned h1[2][4][4];
    {
        unsigned a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int r0 = mt * 16 + g, r1 = r0 + 8;
            a[mt][0] = smw[(r0 * JK_RT_NINP + 2 * t) >> 1];
            a[mt][1] = smw[(r1 * JK_RT_NINP + 2 * t) >> 1];
            a[mt][2] = smw[(r0 * JK_RT_NINP + 2 * t + 8) >> 1];
            a[mt][3] = smw[(r1 * JK_RT_NINP + 2 * t + 8) >> 1];
        }
        // layer 1: 16 -> 64, bias in the accumulator, ReLU, BF16 -> A of layer 2
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const uint2 b = __ldg(W1 + nt * 32 + lane);
            const float bl = __ldg(&R->b1[nt * 8 + 2 * t]), bh = __ldg(&R->b1[nt * 8 + 2 * t + 1]);
            const int ks = nt >> 1, half = nt & 1;
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                float c[4] = {bl, bh, bl, bh};
                jk_mma_bf16(c, a[mt], b.x, b.y);
                // A fragments of layer 2 for k-step ks: {rows g: cols 2t..} = h1[ks][0],
                // {g+8} = h1[ks][1], {g, +8 cols} = h1[ks][2], {g+8, +8} = h1[ks][3]
                h1[mt][ks][half * 2 + 0] = jk_pack_bf16(fmaxf(c[0], 0.0f), fmaxf(c[1], 0.0f));
                h1[mt][ks][half * 2 + 1] = jk_pack_bf16(fmaxf(c[2], 0.0f), fmaxf(c[3], 0.0f));
            }
        }
    }
    // layers 2 and 3: layer-3 k-step k3 takes layer-2 n-tiles 2 k3 and 2 k3 + 1
    float o[2][4] = {{0.0f, 0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f, 0.0f}};
#pragma unroll
    for (int k3 = 0; k3 < 4; ++k3) {
        unsigned a3[2][4];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int nt = 2 * k3 + half;
            const float bl = __ldg(&R->b2[nt * 8 + 2 * t]), bh = __ldg(&R->b2[nt * 8 + 2 * t + 1]);
            float c[2][4] = {{bl, bh, bl, bh}, {bl, bh, bl, bh}};
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint2 b = __ldg(W2 + (ks * 8 + nt) * 32 + lane);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) jk_mma_bf16(c[mt], h1[mt][ks], b.x, b.y);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                a3[mt][half * 2 + 0] = jk_pack_bf16(fmaxf(c[mt][0], 0.0f), fmaxf(c[mt][1], 0.0f));
                a3[mt][half * 2 + 1] = jk_pack_bf16(fmaxf(c[mt][2], 0.0f), fmaxf(c[mt][3], 0.0f));
            }
        }
        // layer 3: 64 -> 1 (an 8-wide n-tile, column 0 used)
        const uint2 b = __ldg(W3 + k3 * 32 + lane);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) jk_mma_bf16(o[mt], a3[mt], b.x, b.y);
    }
    float out[2][2];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        out[mt][0] = o[mt][0];
        out[mt][1] = o[mt][2];
    }
    __syncwarp();
    // row r of tile mt sits in lane 4 (r % 8), register c0 (r < 8) or c2
    const int mt = lane >> 4, rr = lane & 15, src = 4 * (rr & 7);
    const float v00 = __shfl_sync(0xffffffffu, out[0][0], src);
    const float v01 = __shfl_sync(0xffffffffu, out[0][1], src);
    const float v10 = __shfl_sync(0xffffffffu, out[1][0], src);
    const float v11 = __shfl_sync(0xffffffffu, out[1][1], src);
    const float y = mt == 0 ? (rr < 8 ? v00 : v01) : (rr < 8 ? v10 : v11);
    return __fadd_rn(__fadd_rn(y, __ldg(&R->b3)), __ldg(&R->margin));
}

// FP32 route decisions for the band candidates of a warp (warp-synchronous).
__device__ __forceinline__ bool jk_router_to_fp32_warp(const JkRouterDev *__restrict__ R, const JkPairFeat &fa,
                                                       const JkPairFeat &fc, float B, float dmax, float tau,
                                                       unsigned short *sm)
{
    float x[JK_RT_NIN];
    jk_router_features(fa, fc, B, dmax, tau, x);
    const float y = jk_router_warp(R, x, sm);
    return __fadd_rn(x[11], y) <= 0.0f;
}
