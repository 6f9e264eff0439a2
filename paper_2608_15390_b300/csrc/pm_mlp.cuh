// pm_mlp.cuh -- the learned proposal's network (8 -> 64 -> 64 -> 1, tanh-GELU) on
// BF16 tensor cores with FP32 accumulation, and its binary32 score exponent.
//
// Training: a 16-row tile goes through the three layers as mma.sync.m16n8k16
// operations; the FP32 accumulator fragments of one layer become the BF16 A
// fragments of the next without leaving registers (the accumulator of n-tiles
// 2k, 2k+1 is exactly the A fragment of k-tile k).  Inference inside the
// trajectory kernel runs transposed (hidden units x 8 candidates, see
// mlp_infer8).  Weights sit in shared memory in the [out][in] row-major
// layout, so every B fragment is one 32-bit load and every A fragment of the
// transposed form one ldmatrix.
#pragma once
#include <cuda_bf16.h>
#include "pm_device.cuh"

namespace pm {

constexpr int kNF = 8, kNH = 64;
constexpr int kNParam = kNH * kNF + kNH + kNH * kNH + kNH + kNH + 1;  // 4801

// Row strides (in bf16 elements) of the weights in shared memory: 24 and 72
// put the 8 row groups of a fragment load in distinct banks (a 16- or
// 64-element stride would map all of them to the same bank).
constexpr int kW1S = 24, kWS = 72, kFS = 24;

// device image of a model; the first kModelInferBytes are what inference needs
struct DevModel {
    uint16_t w1p[kNH * kW1S];  // W1 [out][in], in padded 8 -> 16 with zeros (stride 24)
    uint16_t w2[kNH * kWS];    // W2 [out][in] (stride 72)
    uint16_t w3p[8 * kWS];     // row 0 = W3, rows 1..7 zero (an 8-wide n-tile)
    float b1[kNH];
    float b2[kNH];
    float b3[4];
    uint16_t w2t[kNH * kWS];   // W2 transposed [in][out] (training only)
};
constexpr int kModelInferBytes =
    (int)(sizeof(uint16_t) * (kNH * kW1S + kNH * kWS + 8 * kWS) + sizeof(float) * (2 * kNH + 4));

__device__ __forceinline__ uint32_t ld32(const uint16_t* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// GELU in its tanh form, g(x) = x/2 (1 + tanh(c (x + a x^3))), c = sqrt(2/pi),
// a = 0.044715, with the hardware tanh approximation (about 2^-11 relative)
__device__ __forceinline__ float tanh_hw(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float gelu_f(float x)
{
    const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
    return 0.5f * x * (1.0f + tanh_hw(u));
}
// both at once, from one tanh
__device__ __forceinline__ void gelu_fd(float x, float& g, float& gd)
{
    const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
    const float th = tanh_hw(u);
    g = 0.5f * x * (1.0f + th);
    gd = 0.5f * (1.0f + th) + 0.5f * x * (1.0f - th * th) * 0.7978845608028654f * (1.0f + 0.134145f * x * x);
}
__device__ __forceinline__ float gelu_d(float x)
{
    const float u = 0.7978845608028654f * (x + 0.044715f * x * x * x);
    const float th = tanh_hw(u);
    return 0.5f * (1.0f + th) + 0.5f * x * (1.0f - th * th) * 0.7978845608028654f * (1.0f + 0.134145f * x * x);
}

// e^x of the learned proposal's score: x clamped to [-20, 20] (NaN -> -20),
// 2^(x log2 e) with a degree-7 Taylor polynomial of 2^f = e^(f ln 2) on
// |f| <= 1/2; coefficients (ln 2)^k / k! and log2 e rounded to binary32, every
// operation correctly rounded (the CPU oracle computes the same bits).
__device__ __forceinline__ float exp_score(float x)
{
    if (!(x >= -20.0f)) x = -20.0f;
    if (x > 20.0f) x = 20.0f;
    const float y = __fmul_rn(x, 0x1.715476p+0f);
    const float nn = rintf(y);
    const float f = __fsub_rn(y, nn);
    float p = 0x1.ffcbfcp-17f;
    p = __fadd_rn(__fmul_rn(p, f), 0x1.430912p-13f);
    p = __fadd_rn(__fmul_rn(p, f), 0x1.5d87fep-10f);
    p = __fadd_rn(__fmul_rn(p, f), 0x1.3b2ab6p-7f);
    p = __fadd_rn(__fmul_rn(p, f), 0x1.c6b08ep-5f);
    p = __fadd_rn(__fmul_rn(p, f), 0x1.ebfbe0p-3f);
    p = __fadd_rn(__fmul_rn(p, f), 0x1.62e430p-1f);
    p = __fadd_rn(__fmul_rn(p, f), 1.0f);
    return __fmul_rn(p, __int_as_float((127 + (int)nn) << 23));
}

// Forward of one 16-row tile whose features are A fragment `a` (bf16, K = 16
// with features 8..15 zero).  Returns the outputs of rows g and g + 8 in lanes
// with (lane & 3) == 0 (g = lane >> 2).  If z1 / z2 are given, the FP32
// pre-activations of both hidden layers are kept (accumulator layout,
// [n-tile][4]) for the backward pass, and h1 the BF16 A fragments of layer 2.
struct FwdKeep {
    float z1[8][4];
    float z2[8][4];
    uint32_t h1[4][4];
    uint32_t h2[4][4];
};

template <bool KEEP>
__device__ __forceinline__ void mlp_fwd_tile(const DevModel* M, const uint32_t (&a)[4], int lane, float& y_lo,
                                             float& y_hi, FwdKeep* keep)
{
    const int g = lane >> 2, t = lane & 3;
    uint32_t h[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        float acc[2][4];
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            const int j = 2 * kk + jj;
            const float c0 = M->b1[8 * j + 2 * t], c1 = M->b1[8 * j + 2 * t + 1];
            acc[jj][0] = c0; acc[jj][1] = c1; acc[jj][2] = c0; acc[jj][3] = c1;
            mma16816(acc[jj], a, ld32(M->w1p + (8 * j + g) * kW1S + 2 * t), ld32(M->w1p + (8 * j + g) * kW1S + 2 * t + 8));
            if (KEEP) {
#pragma unroll
                for (int q = 0; q < 4; ++q) keep->z1[j][q] = acc[jj][q];
            }
        }
        h[kk][0] = pack_bf16(gelu_f(acc[0][0]), gelu_f(acc[0][1]));
        h[kk][1] = pack_bf16(gelu_f(acc[0][2]), gelu_f(acc[0][3]));
        h[kk][2] = pack_bf16(gelu_f(acc[1][0]), gelu_f(acc[1][1]));
        h[kk][3] = pack_bf16(gelu_f(acc[1][2]), gelu_f(acc[1][3]));
        if (KEEP) {
#pragma unroll
            for (int q = 0; q < 4; ++q) keep->h1[kk][q] = h[kk][q];
        }
    }
    uint32_t h2[4][4];
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
        float acc[2][4];
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
            const int j = 2 * k2 + jj;
            const float c0 = M->b2[8 * j + 2 * t], c1 = M->b2[8 * j + 2 * t + 1];
            acc[jj][0] = c0; acc[jj][1] = c1; acc[jj][2] = c0; acc[jj][3] = c1;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma16816(acc[jj], h[kk], ld32(M->w2 + (8 * j + g) * kWS + 16 * kk + 2 * t),
                         ld32(M->w2 + (8 * j + g) * kWS + 16 * kk + 2 * t + 8));
            if (KEEP) {
#pragma unroll
                for (int q = 0; q < 4; ++q) keep->z2[j][q] = acc[jj][q];
            }
        }
        h2[k2][0] = pack_bf16(gelu_f(acc[0][0]), gelu_f(acc[0][1]));
        h2[k2][1] = pack_bf16(gelu_f(acc[0][2]), gelu_f(acc[0][3]));
        h2[k2][2] = pack_bf16(gelu_f(acc[1][0]), gelu_f(acc[1][1]));
        h2[k2][3] = pack_bf16(gelu_f(acc[1][2]), gelu_f(acc[1][3]));
        if (KEEP) {
#pragma unroll
            for (int q = 0; q < 4; ++q) keep->h2[k2][q] = h2[k2][q];
        }
    }
    float acc3[4];
    acc3[0] = (t == 0) ? M->b3[0] : 0.0f;
    acc3[1] = 0.0f;
    acc3[2] = acc3[0];
    acc3[3] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
        mma16816(acc3, h2[kk], ld32(M->w3p + g * kWS + 16 * kk + 2 * t), ld32(M->w3p + g * kWS + 16 * kk + 2 * t + 8));
    y_lo = acc3[0];
    y_hi = acc3[2];
}

// 8x8 transpose of a bf16 fragment (row lane/4, columns 2(lane%4), +1)
__device__ __forceinline__ uint32_t trans8x8(uint32_t x)
{
    uint32_t y;
    asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;\n" : "=r"(y) : "r"(x));
    return y;
}

// A fragment (16 x 16 bf16, row-major with stride kWS) of shared memory by one
// ldmatrix.x4: lane l supplies row (l & 7) + 8 ((l >> 3) & 1), column
// 8 (l >> 4); the four 8x8 matrices come back as a0..a3 of mma.m16n8k16
__device__ __forceinline__ void ldsm_a(uint32_t (&a)[4], const uint16_t* tile, int lane)
{
    const uint16_t* p = tile + ((lane & 7) + 8 * ((lane >> 3) & 1)) * kWS + 8 * (lane >> 4);
    const uint32_t addr = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3])
                 : "r"(addr));
}

// Inference for up to 8 candidates, transposed: the hidden units are the M
// dimension (four 16-row m-tiles) and the candidates the N dimension (8), so
// a minimum-degree step, which has 2 or 3 live candidates most of the time,
// pays for 8 columns instead of a 16-row tile.  Features are rows 0..7 of
// `feat` (bf16 [8][kFS], model and features in shared memory).  An
// accumulator fragment of hidden units x candidates, packed to bf16 and
// transposed 8x8 by movmatrix, is exactly the B fragment of the next layer
// (and the A fragment of the output layer).  Returns the output of candidate
// lane >> 2 in lanes with (lane & 3) == 0.
__device__ __forceinline__ float mlp_infer8(const DevModel* M, const uint16_t* feat, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    const uint32_t xb = ld32(feat + g * kFS + 2 * t);  // features 2t, 2t+1 of candidate g
    uint32_t hb[4][2];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
        const int h0 = 16 * mt + g;
        float acc[4] = {M->b1[h0], M->b1[h0], M->b1[h0 + 8], M->b1[h0 + 8]};
        const uint32_t a[4] = {ld32(M->w1p + h0 * kW1S + 2 * t), ld32(M->w1p + (h0 + 8) * kW1S + 2 * t), 0u, 0u};
        mma16816(acc, a, xb, 0u);
        hb[mt][0] = trans8x8(pack_bf16(gelu_f(acc[0]), gelu_f(acc[1])));
        hb[mt][1] = trans8x8(pack_bf16(gelu_f(acc[2]), gelu_f(acc[3])));
    }
    float acc3[4] = {t == 0 ? M->b3[0] : 0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
    for (int mt = 0; mt < 4; ++mt) {
        const int h0 = 16 * mt + g;
        float acc[4] = {M->b2[h0], M->b2[h0], M->b2[h0 + 8], M->b2[h0 + 8]};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t a[4];
            ldsm_a(a, M->w2 + 16 * mt * kWS + 16 * kk, lane);
            mma16816(acc, a, hb[kk][0], hb[kk][1]);
        }
        // output layer: rows = candidates (8 of 16 used), k = these 16 hidden units
        const uint32_t a3[4] = {trans8x8(pack_bf16(gelu_f(acc[0]), gelu_f(acc[1]))), 0u,
                                trans8x8(pack_bf16(gelu_f(acc[2]), gelu_f(acc[3]))), 0u};
        mma16816(acc3, a3, ld32(M->w3p + g * kWS + 16 * mt + 2 * t), ld32(M->w3p + g * kWS + 16 * mt + 2 * t + 8));
    }
    return acc3[0];
}

}  // namespace pm
