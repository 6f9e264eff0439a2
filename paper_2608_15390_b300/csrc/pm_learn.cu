// pm_learn.cu -- training of the learned proposal (an extension:
// the paper has no learned part).  Forward and backward run on BF16 tensor
// cores (mma.sync.m16n8k16, FP32 accumulation); Adam keeps FP32 master
// weights and refreshes the BF16 device image after every step.
//
// Losses on the recorded (features, target) pairs, target = the SK scale
// product ln(r_v c_l): the mean squared error, or the per-step centred squared
// error, which removes each step's mean residual first (the proposal of Eq. 3
// normalises a step's scores, so a step-wide offset of the logits is
// invisible to it).  For the latter a forward pass writes the residuals of
// the batch, and the backward kernel reads its group's mean from them.
#include <cmath>
#include "pm_mlp.cuh"

namespace pm {

namespace {

constexpr int kTrainWarps = 4;
constexpr int kTrainRows = 32 * kTrainWarps;  // rows per CTA iteration

// offsets of the flat parameter vector: W1[64][8], b1, W2[64][64], b2, W3, b3
constexpr int oW1 = 0, oB1 = kNH * kNF, oW2 = oB1 + kNH, oB2 = oW2 + kNH * kNH, oW3 = oB2 + kNH, oB3 = oW3 + kNH;

__device__ __forceinline__ float bf16lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }
__device__ __forceinline__ uint16_t bf16_bits(float x)
{
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t*>(&b);
}

// sum over the 8 lanes sharing (lane & 3)
__device__ __forceinline__ float sum_over_g(float v)
{
    v += __shfl_xor_sync(kFull, v, 4);
    v += __shfl_xor_sync(kFull, v, 8);
    v += __shfl_xor_sync(kFull, v, 16);
    return v;
}

struct TrainSmem {
    DevModel M;
    uint16_t dz2t[kNH * kTrainRows];  // [out][row]
    uint16_t h1t[kNH * kTrainRows];   // [in][row]
    uint16_t dz1t[kNH * kTrainRows];  // [out][row]
    uint16_t xt[8 * kTrainRows];      // [feature][row]
};

// Gradient of the loss over rows perm[row0 .. row0 + B) of (feat, target),
// accumulated into grad[kNParam] (FP32 atomics) and loss.  resid == nullptr:
// mean squared error.  Otherwise the centred loss: resid[r] is the residual
// of batch row r (from mlp_resid_kernel, the same forward), group[] the group
// code of a pair (index within its step << 16 | the step's pair count), and
// the rows of a step are consecutive in the batch.
__global__ void __launch_bounds__(kTrainWarps * 32) mlp_grad_kernel(const DevModel* Mg, const float* feat,
                                                                    const float* target, const int* perm,
                                                                    int64_t row0, int B, float inv_b,
                                                                    const float* resid, const uint32_t* group,
                                                                    float* part, double* loss_part)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5, g = lane >> 2, t = lane & 3;
    {
        const uint4* src = reinterpret_cast<const uint4*>(Mg);
        uint4* dst = reinterpret_cast<uint4*>(&S.M);
        for (int q = tid; q < (int)(sizeof(DevModel) / 16); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    const DevModel* M = &S.M;
    float acc_w2[8][4], acc_w1[4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
        for (int q = 0; q < 4; ++q) acc_w2[j][q] = 0.0f;
    for (int q = 0; q < 4; ++q) acc_w1[q] = 0.0f;
    float acc_b1[16], acc_b2[16], acc_w3[16];
    for (int q = 0; q < 16; ++q) acc_b1[q] = acc_b2[q] = acc_w3[q] = 0.0f;
    float acc_b3 = 0.0f;
    double loss = 0.0;

    const int iters = (B + kTrainRows - 1) / kTrainRows;
    for (int it = blockIdx.x; it < iters; it += gridDim.x) {
#pragma unroll 1
        for (int mt = 0; mt < 2; ++mt) {
            const int lr0 = 32 * w + 16 * mt;              // local row of this tile
            const int r_g = it * kTrainRows + lr0 + g;     // batch rows g, g + 8
            const int r_g8 = r_g + 8;
            const bool v_g = r_g < B, v_g8 = r_g8 < B;
            float x_g[2] = {0.f, 0.f}, x_g8[2] = {0.f, 0.f};
            float t_g = 0.f, t_g8 = 0.f;
            if (v_g) {
                const int64_t src = perm[row0 + r_g];
                x_g[0] = feat[src * kNF + 2 * t];
                x_g[1] = feat[src * kNF + 2 * t + 1];
                t_g = target[src];
            }
            if (v_g8) {
                const int64_t src = perm[row0 + r_g8];
                x_g8[0] = feat[src * kNF + 2 * t];
                x_g8[1] = feat[src * kNF + 2 * t + 1];
                t_g8 = target[src];
            }
            uint32_t a[4] = {pack_bf16(x_g[0], x_g[1]), pack_bf16(x_g8[0], x_g8[1]), 0u, 0u};
            S.xt[(2 * t) * kTrainRows + lr0 + g] = (uint16_t)(a[0] & 0xFFFFu);
            S.xt[(2 * t + 1) * kTrainRows + lr0 + g] = (uint16_t)(a[0] >> 16);
            S.xt[(2 * t) * kTrainRows + lr0 + g + 8] = (uint16_t)(a[1] & 0xFFFFu);
            S.xt[(2 * t + 1) * kTrainRows + lr0 + g + 8] = (uint16_t)(a[1] >> 16);
            FwdKeep K;
            float y_lo, y_hi;
            mlp_fwd_tile<true>(M, a, lane, y_lo, y_hi, &K);
            // h1 -> shared [in][row]
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int c = 16 * kk + 2 * t;
                S.h1t[c * kTrainRows + lr0 + g] = (uint16_t)(K.h1[kk][0] & 0xFFFFu);
                S.h1t[(c + 1) * kTrainRows + lr0 + g] = (uint16_t)(K.h1[kk][0] >> 16);
                S.h1t[c * kTrainRows + lr0 + g + 8] = (uint16_t)(K.h1[kk][1] & 0xFFFFu);
                S.h1t[(c + 1) * kTrainRows + lr0 + g + 8] = (uint16_t)(K.h1[kk][1] >> 16);
                S.h1t[(c + 8) * kTrainRows + lr0 + g] = (uint16_t)(K.h1[kk][2] & 0xFFFFu);
                S.h1t[(c + 9) * kTrainRows + lr0 + g] = (uint16_t)(K.h1[kk][2] >> 16);
                S.h1t[(c + 8) * kTrainRows + lr0 + g + 8] = (uint16_t)(K.h1[kk][3] & 0xFFFFu);
                S.h1t[(c + 9) * kTrainRows + lr0 + g + 8] = (uint16_t)(K.h1[kk][3] >> 16);
            }
            // output gradient dL/dy = 2 e / B, e the (centred) residual
            auto centred = [&](int r) -> float {
                const uint32_t code = group[perm[row0 + r]];
                const int q = (int)(code >> 16), size = (int)(code & 0xFFFFu);
                float mean = 0.f;
                for (int k = 0; k < size; ++k) mean += resid[r - q + k];
                return resid[r] - mean / (float)size;
            };
            float dy_lo = 0.f, dy_hi = 0.f;
            if (t == 0) {
                if (v_g) {
                    const float e = resid ? centred(r_g) : y_lo - t_g;
                    dy_lo = 2.f * e * inv_b;
                    loss += (double)e * e * inv_b;
                }
                if (v_g8) {
                    const float e = resid ? centred(r_g8) : y_hi - t_g8;
                    dy_hi = 2.f * e * inv_b;
                    loss += (double)e * e * inv_b;
                }
                acc_b3 += dy_lo + dy_hi;
            }
            dy_lo = __shfl_sync(kFull, dy_lo, g * 4);
            dy_hi = __shfl_sync(kFull, dy_hi, g * 4);
            // dW3 and dz2 = dy W3 gelu'(z2)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float p0 = dy_lo * bf16lo(K.h2[kk][0]) + dy_hi * bf16lo(K.h2[kk][1]);
                const float p1 = dy_lo * bf16hi(K.h2[kk][0]) + dy_hi * bf16hi(K.h2[kk][1]);
                const float p2 = dy_lo * bf16lo(K.h2[kk][2]) + dy_hi * bf16lo(K.h2[kk][3]);
                const float p3 = dy_lo * bf16hi(K.h2[kk][2]) + dy_hi * bf16hi(K.h2[kk][3]);
                acc_w3[4 * kk + 0] += sum_over_g(p0);
                acc_w3[4 * kk + 1] += sum_over_g(p1);
                acc_w3[4 * kk + 2] += sum_over_g(p2);
                acc_w3[4 * kk + 3] += sum_over_g(p3);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = 8 * j + 2 * t;
                const uint32_t w3pair = ld32(M->w3p + c);  // row 0 of w3p holds W3
                const float w3a = bf16lo(w3pair), w3b = bf16hi(w3pair);
                K.z2[j][0] = dy_lo * w3a * gelu_d(K.z2[j][0]);
                K.z2[j][1] = dy_lo * w3b * gelu_d(K.z2[j][1]);
                K.z2[j][2] = dy_hi * w3a * gelu_d(K.z2[j][2]);
                K.z2[j][3] = dy_hi * w3b * gelu_d(K.z2[j][3]);
                acc_b2[2 * j] += sum_over_g(K.z2[j][0] + K.z2[j][2]);
                acc_b2[2 * j + 1] += sum_over_g(K.z2[j][1] + K.z2[j][3]);
                S.dz2t[c * kTrainRows + lr0 + g] = bf16_bits(K.z2[j][0]);
                S.dz2t[(c + 1) * kTrainRows + lr0 + g] = bf16_bits(K.z2[j][1]);
                S.dz2t[c * kTrainRows + lr0 + g + 8] = bf16_bits(K.z2[j][2]);
                S.dz2t[(c + 1) * kTrainRows + lr0 + g + 8] = bf16_bits(K.z2[j][3]);
            }
            // dh1 = dz2 W2 (tensor cores), dz1 = dh1 gelu'(z1)
            uint32_t da[4][4];
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                da[kk][0] = pack_bf16(K.z2[2 * kk][0], K.z2[2 * kk][1]);
                da[kk][1] = pack_bf16(K.z2[2 * kk][2], K.z2[2 * kk][3]);
                da[kk][2] = pack_bf16(K.z2[2 * kk + 1][0], K.z2[2 * kk + 1][1]);
                da[kk][3] = pack_bf16(K.z2[2 * kk + 1][2], K.z2[2 * kk + 1][3]);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma16816(d, da[kk], ld32(M->w2t + (8 * j + g) * kWS + 16 * kk + 2 * t),
                             ld32(M->w2t + (8 * j + g) * kWS + 16 * kk + 2 * t + 8));
                const int c = 8 * j + 2 * t;
                const float z0 = d[0] * gelu_d(K.z1[j][0]), z1 = d[1] * gelu_d(K.z1[j][1]);
                const float z2 = d[2] * gelu_d(K.z1[j][2]), z3 = d[3] * gelu_d(K.z1[j][3]);
                acc_b1[2 * j] += sum_over_g(z0 + z2);
                acc_b1[2 * j + 1] += sum_over_g(z1 + z3);
                S.dz1t[c * kTrainRows + lr0 + g] = bf16_bits(z0);
                S.dz1t[(c + 1) * kTrainRows + lr0 + g] = bf16_bits(z1);
                S.dz1t[c * kTrainRows + lr0 + g + 8] = bf16_bits(z2);
                S.dz1t[(c + 1) * kTrainRows + lr0 + g + 8] = bf16_bits(z3);
            }
        }
        __syncthreads();
        // weight gradients over the CTA's 128 rows: warp w owns output rows 16w..16w+15
#pragma unroll 1
        for (int kt = 0; kt < kTrainRows / 16; ++kt) {
            const uint16_t* A2 = S.dz2t + (16 * w + g) * kTrainRows + 16 * kt + 2 * t;
            uint32_t a2[4] = {ld32(A2), ld32(A2 + 8 * kTrainRows), ld32(A2 + 8), ld32(A2 + 8 * kTrainRows + 8)};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint16_t* Bp = S.h1t + (8 * j + g) * kTrainRows + 16 * kt + 2 * t;
                mma16816(acc_w2[j], a2, ld32(Bp), ld32(Bp + 8));
            }
            const uint16_t* A1 = S.dz1t + (16 * w + g) * kTrainRows + 16 * kt + 2 * t;
            uint32_t a1[4] = {ld32(A1), ld32(A1 + 8 * kTrainRows), ld32(A1 + 8), ld32(A1 + 8 * kTrainRows + 8)};
            const uint16_t* Bx = S.xt + g * kTrainRows + 16 * kt + 2 * t;
            mma16816(acc_w1, a1, ld32(Bx), ld32(Bx + 8));
        }
        __syncthreads();
    }
    // flush into this CTA's row of partial sums (a fixed-order reduction over
    // the CTAs follows, so the gradient does not depend on scheduling): the
    // weight entries belong to one lane each, the bias and W3 entries of the
    // four warps are added in warp order through shared memory
    float* prow = part + (size_t)blockIdx.x * kNParam;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int row = 16 * w + g, col = 8 * j + 2 * t;
        prow[oW2 + row * kNH + col] = acc_w2[j][0];
        prow[oW2 + row * kNH + col + 1] = acc_w2[j][1];
        prow[oW2 + (row + 8) * kNH + col] = acc_w2[j][2];
        prow[oW2 + (row + 8) * kNH + col + 1] = acc_w2[j][3];
    }
    {
        const int row = 16 * w + g, col = 2 * t;
        prow[oW1 + row * kNF + col] = acc_w1[0];
        prow[oW1 + row * kNF + col + 1] = acc_w1[1];
        prow[oW1 + (row + 8) * kNF + col] = acc_w1[2];
        prow[oW1 + (row + 8) * kNF + col + 1] = acc_w1[3];
    }
    float* red = reinterpret_cast<float*>(S.dz2t);  // [kTrainWarps][3 * kNH + 1], free after the last iteration
    double* lred = reinterpret_cast<double*>(S.h1t);
    constexpr int kRed = 3 * kNH + 1;
    if (g == 0) {
        for (int j = 0; j < 8; ++j) {
            red[w * kRed + 8 * j + 2 * t] = acc_b1[2 * j];
            red[w * kRed + 8 * j + 2 * t + 1] = acc_b1[2 * j + 1];
            red[w * kRed + kNH + 8 * j + 2 * t] = acc_b2[2 * j];
            red[w * kRed + kNH + 8 * j + 2 * t + 1] = acc_b2[2 * j + 1];
        }
        for (int kk = 0; kk < 4; ++kk) {
            red[w * kRed + 2 * kNH + 16 * kk + 2 * t] = acc_w3[4 * kk + 0];
            red[w * kRed + 2 * kNH + 16 * kk + 2 * t + 1] = acc_w3[4 * kk + 1];
            red[w * kRed + 2 * kNH + 16 * kk + 8 + 2 * t] = acc_w3[4 * kk + 2];
            red[w * kRed + 2 * kNH + 16 * kk + 8 + 2 * t + 1] = acc_w3[4 * kk + 3];
        }
    }
    if (t == 0) {
        float b3 = acc_b3;
        b3 += __shfl_xor_sync(0x11111111u, b3, 4);
        b3 += __shfl_xor_sync(0x11111111u, b3, 8);
        b3 += __shfl_xor_sync(0x11111111u, b3, 16);
        if (g == 0) red[w * kRed + 3 * kNH] = b3;
    }
    for (int o = 16; o; o >>= 1) loss += __shfl_xor_sync(kFull, loss, o);
    if (lane == 0) lred[w] = loss;
    __syncthreads();
    for (int i = tid; i < kRed; i += blockDim.x) {
        float v = 0.f;
        for (int q = 0; q < kTrainWarps; ++q) v += red[q * kRed + i];
        const int dst = i < kNH ? oB1 + i : i < 2 * kNH ? oB2 + (i - kNH) : i < 3 * kNH ? oW3 + (i - 2 * kNH) : oB3;
        prow[dst] = v;
    }
    if (tid == 0) {
        double l = 0.0;
        for (int q = 0; q < kTrainWarps; ++q) l += lred[q];
        loss_part[blockIdx.x] = l;
    }
}

// grad[i] = sum over the CTAs (in CTA order) of their partial sums; loss alike
__global__ void grad_reduce_kernel(const float* part, const double* loss_part, int ctas, float* grad, double* loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kNParam) {
        float v = 0.f;
        for (int c = 0; c < ctas; ++c) v += part[(size_t)c * kNParam + i];
        grad[i] = v;
    }
    if (i == 0) {
        double l = 0.0;
        for (int c = 0; c < ctas; ++c) l += loss_part[c];
        *loss = l;
    }
}

// outputs of rows 0 .. B-1 of feat (one warp per 16-row tile)
__global__ void __launch_bounds__(128) mlp_forward_kernel(const DevModel* Mg, const float* feat, int B, float* out)
{
    __shared__ __align__(16) uint8_t mraw[kModelInferBytes + 16];
    DevModel* M = reinterpret_cast<DevModel*>(mraw);
    {
        const uint4* src = reinterpret_cast<const uint4*>(Mg);
        uint4* dst = reinterpret_cast<uint4*>(mraw);
        for (int q = threadIdx.x; q < (kModelInferBytes + 15) / 16; q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 16 < B; tile += warps) {
        const int r0 = tile * 16 + g, r1 = r0 + 8;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f;
        if (r0 < B) { x0 = feat[(int64_t)r0 * kNF + 2 * t]; x1 = feat[(int64_t)r0 * kNF + 2 * t + 1]; }
        if (r1 < B) { x2 = feat[(int64_t)r1 * kNF + 2 * t]; x3 = feat[(int64_t)r1 * kNF + 2 * t + 1]; }
        uint32_t a[4] = {pack_bf16(x0, x1), pack_bf16(x2, x3), 0u, 0u};
        float ylo, yhi;
        mlp_fwd_tile<false>(M, a, lane, ylo, yhi, nullptr);
        if (t == 0) {
            if (r0 < B) out[r0] = ylo;
            if (r1 < B) out[r1] = yhi;
        }
    }
}

// residuals y - target of rows perm[row0 .. row0 + B) (one warp per 16-row
// tile), the forward of mlp_grad_kernel without its bookkeeping
__global__ void __launch_bounds__(128) mlp_resid_kernel(const DevModel* Mg, const float* feat, const float* target,
                                                        const int* perm, int64_t row0, int B, float* resid)
{
    __shared__ __align__(16) uint8_t mraw[kModelInferBytes + 16];
    DevModel* M = reinterpret_cast<DevModel*>(mraw);
    {
        const uint4* src = reinterpret_cast<const uint4*>(Mg);
        uint4* dst = reinterpret_cast<uint4*>(mraw);
        for (int q = threadIdx.x; q < (kModelInferBytes + 15) / 16; q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int tile = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 16 < B; tile += warps) {
        const int r0 = tile * 16 + g, r1 = r0 + 8;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f, x3 = 0.f;
        int64_t s0 = 0, s1 = 0;
        if (r0 < B) {
            s0 = perm[row0 + r0];
            x0 = feat[s0 * kNF + 2 * t];
            x1 = feat[s0 * kNF + 2 * t + 1];
        }
        if (r1 < B) {
            s1 = perm[row0 + r1];
            x2 = feat[s1 * kNF + 2 * t];
            x3 = feat[s1 * kNF + 2 * t + 1];
        }
        uint32_t a[4] = {pack_bf16(x0, x1), pack_bf16(x2, x3), 0u, 0u};
        float ylo, yhi;
        mlp_fwd_tile<false>(M, a, lane, ylo, yhi, nullptr);
        if (t == 0) {
            if (r0 < B) resid[r0] = ylo - target[s0];
            if (r1 < B) resid[r1] = yhi - target[s1];
        }
    }
}

// Adam on the FP32 master weights, then the BF16 device image
__global__ void adam_kernel(float* master, float* m1, float* m2, const float* grad, float lr, float b1, float b2,
                            float eps, float c1, float c2, DevModel* img)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParam) return;
    const float gr = grad[i];
    const float mm = b1 * m1[i] + (1.f - b1) * gr;
    const float vv = b2 * m2[i] + (1.f - b2) * gr * gr;
    m1[i] = mm;
    m2[i] = vv;
    const float p = master[i] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    master[i] = p;
    const uint16_t bits = bf16_bits(p);
    if (i < oB1) {
        img->w1p[(i / kNF) * kW1S + (i % kNF)] = bits;
    } else if (i < oW2) {
        img->b1[i - oB1] = p;
    } else if (i < oB2) {
        const int k = i - oW2, o = k / kNH, in = k % kNH;
        img->w2[o * kWS + in] = bits;
        img->w2t[in * kWS + o] = bits;
    } else if (i < oW3) {
        img->b2[i - oB2] = p;
    } else if (i < oB3) {
        img->w3p[i - oW3] = bits;
    } else {
        img->b3[0] = p;
    }
}

// BF16 device image of FP32 parameters (padding entries left as zero)
__global__ void image_kernel(const float* master, DevModel* img)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kNParam) return;
    const float p = master[i];
    const uint16_t bits = bf16_bits(p);
    if (i < oB1) img->w1p[(i / kNF) * kW1S + (i % kNF)] = bits;
    else if (i < oW2) img->b1[i - oB1] = p;
    else if (i < oB2) {
        const int k = i - oW2, o = k / kNH, in = k % kNH;
        img->w2[o * kWS + in] = bits;
        img->w2t[in * kWS + o] = bits;
    } else if (i < oW3) img->b2[i - oB2] = p;
    else if (i < oB3) img->w3p[i - oW3] = bits;
    else img->b3[0] = p;
}

}  // namespace

int model_image_bytes() { return (int)sizeof(DevModel); }
int model_infer_bytes() { return kModelInferBytes; }
int model_param_count() { return kNParam; }

cudaError_t launch_model_image(const float* master, void* img, cudaStream_t st)
{
    image_kernel<<<(kNParam + 127) / 128, 128, 0, st>>>(master, reinterpret_cast<DevModel*>(img));
    return cudaGetLastError();
}

size_t mlp_grad_workspace_bytes(int sm_count)
{
    return (size_t)2 * sm_count * (kNParam * sizeof(float) + sizeof(double)) + 256;
}

cudaError_t launch_mlp_grad(const void* img, const float* feat, const float* target, const int* perm, int64_t row0,
                            int B, const uint32_t* group, float* resid, float* grad, double* loss, int sm_count,
                            void* work, cudaStream_t st)
{
    const DevModel* M = reinterpret_cast<const DevModel*>(img);
    if (group) {  // centred loss: the batch's residuals first
        const int tiles = (B + 15) / 16;
        int rg = (tiles + 3) / 4;
        if (rg > 4 * sm_count) rg = 4 * sm_count;
        mlp_resid_kernel<<<rg, 128, 0, st>>>(M, feat, target, perm, row0, B, resid);
    }
    const int smem = (int)sizeof(TrainSmem);
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int iters = (B + kTrainRows - 1) / kTrainRows;
    const int grid = iters < 2 * sm_count ? iters : 2 * sm_count;
    float* part = reinterpret_cast<float*>(work);
    double* loss_part = reinterpret_cast<double*>(
        reinterpret_cast<uint8_t*>(work) + ((size_t)2 * sm_count * kNParam * sizeof(float) + 255) / 256 * 256);
    mlp_grad_kernel<<<grid, kTrainWarps * 32, smem, st>>>(M, feat, target, perm, row0, B, 1.0f / (float)B,
                                                           group ? resid : nullptr, group, part, loss_part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    grad_reduce_kernel<<<(kNParam + 255) / 256, 256, 0, st>>>(part, loss_part, grid, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const void* img, const float* feat, int B, float* out, int sm_count, cudaStream_t st)
{
    const int tiles = (B + 15) / 16;
    int grid = (tiles + 3) / 4;
    if (grid > 4 * sm_count) grid = 4 * sm_count;
    mlp_forward_kernel<<<grid, 128, 0, st>>>(reinterpret_cast<const DevModel*>(img), feat, B, out);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* master, float* m1, float* m2, const float* grad, float lr, float b1, float b2, float eps,
                        int step, void* img, cudaStream_t st)
{
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(kNParam + 127) / 128, 128, 0, st>>>(master, m1, m2, grad, lr, b1, b2, eps, c1, c2,
                                                       reinterpret_cast<DevModel*>(img));
    return cudaGetLastError();
}

}  // namespace pm
