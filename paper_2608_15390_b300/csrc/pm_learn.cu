// pm_learn.cu -- training of the learned proposal (an extension:
// the paper has no learned part).  The gradient's forward and backward run on
// the 5th-generation tensor core (tcgen05 MMAs from shared-memory tiles into
// tensor memory, BF16 operands, FP32 accumulation); the residual pass of the
// centred loss and the standalone forward use mma.sync tiles of the inference
// network; Adam keeps FP32 master weights and refreshes the BF16 device image
// after every step.
//
// Losses on the recorded (features, target) pairs, target = the SK scale
// product ln(r_v c_l): the mean squared error, or the per-step centred squared
// error, which removes each step's mean residual first (the proposal of Eq. 3
// normalises a step's scores, so a step-wide offset of the logits is
// invisible to it).  For the latter a forward pass writes the residuals of
// the batch, and the backward kernel reads its group's mean from them.
#include <cmath>
#include <cstddef>
#include "pm_mlp.cuh"
#include "pm_umma.cuh"

namespace pm {

namespace {

// offsets of the flat parameter vector: W1[64][8], b1, W2[64][64], b2, W3, b3
constexpr int oW1 = 0, oB1 = kNH * kNF, oW2 = oB1 + kNH, oB2 = oW2 + kNH * kNH, oW3 = oB2 + kNH, oB3 = oW3 + kNH;

__device__ __forceinline__ float bf16lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }
__device__ __forceinline__ uint16_t bf16_bits(float x)
{
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t*>(&b);
}

// ---- gradient on the 5th-generation tensor core ----
//
// One CTA of 128 threads (a warpgroup: thread r owns row r of a 128-row
// tile, which is TMEM lane r) runs tiles of the batch.  Per tile, with one
// thread issuing the MMAs into tensor memory and an mbarrier tracking their
// completion:
//   G1  D1 = X W1^T                        (128 x 64, K = 16)
//       h1 = gelu(D1 + b1)                 -> H tile, bf16
//   G2  D2 = h1 W2^T                       (128 x 64, K = 64)
//       z2 = D2 + b2, h2 = gelu(z2), y = h2 . w3 + b3, dy = dL/dy,
//       dz2 = dy w3 gelu'(z2)              -> A tile [dz2 | h2], H tile [.. | 1, dy]
//   G3  D3 = dz2 W2                        (dh1; 128 x 64, K = 64)
//   G4  D4 += [dz2 | h2]^T [h1 | 1 | dy]   (128 x 80, K = the 128 rows)
//       dz1 = D3 gelu'(D1 + b1)            -> B tile [dz1 | 0]
//   G5  D5 += [dz1 | 0]^T [X | 1]          (128 x 16, K = the 128 rows)
// D4 accumulates dW2 (rows 0-63, columns 0-63), db2 (column 64) and dW3
// (rows 64-127, columns 65 + 66: dy split into two bf16 parts); D5 dW1
// (rows 0-63, columns 0-7) and db1 (column 8): the bias and output-layer
// gradients come out of the same MMAs through the constant-one and dy
// columns.  Operands are bf16 (as the mma.sync path had them: features,
// activations, dz), accumulation FP32.
constexpr int kTcRows = 128;
constexpr int kCX = 16, kCH = 80, kCA = 128, kCB = 128;   // columns of the operand tiles
constexpr uint32_t kTmemCols = 256;
constexpr uint32_t kD1 = 0, kD2 = 64, kD4 = 128, kD5 = 208;  // TMEM columns of the accumulators
constexpr uint32_t kWaitPolls = 1u << 24;
constexpr uint16_t kBf16One = 0x3F80;

struct TcSmem {
    uint8_t tX[2][kTcRows * kCX * 2];  // [X | 1 | 0], two tiles (the next tile's G1 overlaps this one's G5)
    uint8_t tH[kTcRows * kCH * 2];   // [h1 | 1, dy_hi, dy_lo, 0 ...]
    uint8_t tA[kTcRows * kCA * 2];   // [dz2 | h2]
    uint8_t tB[kTcRows * kCB * 2];   // [dz1 | 0]
    uint8_t w1[kNH * kCX * 2];       // W1 [hidden][16], inputs 8..15 zero
    uint8_t w2[kNH * kNH * 2];       // W2 [out][in]
    uint64_t mbar;
    uint32_t tmem;
    float b3;
    float b1[kNH], b2[kNH], w3[kNH];
    float red[kTcRows / 32];
    double lred[kTcRows / 32];
};

__device__ __forceinline__ void st_row16(uint8_t* tile, int r, int c0, int C, const uint32_t (&p)[8])
{
    *reinterpret_cast<uint4*>(tile + blk_off(r, c0, C)) = make_uint4(p[0], p[1], p[2], p[3]);
    *reinterpret_cast<uint4*>(tile + blk_off(r, c0 + 8, C)) = make_uint4(p[4], p[5], p[6], p[7]);
}

// Gradient of the loss over rows perm[row0 .. row0 + B) of (feat, target)
// into this CTA's row of partial sums (part[blockIdx.x][kNParam],
// loss_part[blockIdx.x]).  resid == nullptr: mean squared error.  Otherwise
// the centred loss: resid[r] is the residual of batch row r (from
// mlp_resid_kernel), group[] the group code of a pair (index within its step
// << 16 | the step's pair count), and the rows of a step are consecutive in
// the batch.  *err is set if an MMA completion wait runs out.
__global__ void __launch_bounds__(kTcRows) mlp_grad_kernel(const DevModel* Mg, const float* feat,
                                                           const float* target, const int* perm, int64_t row0,
                                                           int B, float inv_b, const float* resid,
                                                           const uint32_t* group, float* part, double* loss_part,
                                                           int* err)
{
    extern __shared__ __align__(128) uint8_t smem_raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = tid;  // tile row and TMEM lane
    {
        uint4* p = reinterpret_cast<uint4*>(smem_raw);
        constexpr int n16 = (int)(offsetof(TcSmem, w1) / 16);
        for (int q = tid; q < n16; q += kTcRows) p[q] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    for (int q = tid; q < kNH * kCX; q += kTcRows) {
        const int h = q / kCX, i = q % kCX;
        *reinterpret_cast<uint16_t*>(S.w1 + blk_off(h, i, kCX)) = i < kNF ? Mg->w1p[h * kW1S + i] : (uint16_t)0;
    }
    for (int q = tid; q < kNH * kNH; q += kTcRows) {
        const int o = q / kNH, i = q % kNH;
        *reinterpret_cast<uint16_t*>(S.w2 + blk_off(o, i, kNH)) = Mg->w2[o * kWS + i];
    }
    for (int q = tid; q < kNH; q += kTcRows) {
        S.b1[q] = Mg->b1[q];
        S.b2[q] = Mg->b2[q];
        S.w3[q] = __uint_as_float((uint32_t)Mg->w3p[q] << 16);
    }
    *reinterpret_cast<uint16_t*>(S.tX[0] + blk_off(r, kNF, kCX)) = kBf16One;
    *reinterpret_cast<uint16_t*>(S.tX[1] + blk_off(r, kNF, kCX)) = kBf16One;
    *reinterpret_cast<uint16_t*>(S.tH + blk_off(r, kNH, kCH)) = kBf16One;
    if (tid == 0) {
        S.b3 = Mg->b3[0];
        mbar_init(&S.mbar, 1);
    }
    if (warp == 0) tmem_alloc(&S.tmem, kTmemCols);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's TMEM lanes
    const uint32_t aX0 = smem_addr(S.tX[0]), aH = smem_addr(S.tH), aA = smem_addr(S.tA), aB = smem_addr(S.tB),
                   aW1 = smem_addr(S.w1), aW2 = smem_addr(S.w2);
    const uint32_t id64 = umma_idesc_bf16(128, 64, 0, 0), id3 = umma_idesc_bf16(128, 64, 0, 1),
                   id4 = umma_idesc_bf16(128, 80, 1, 1), id5 = umma_idesc_bf16(128, 16, 1, 1);
    uint32_t phase = 0;
    bool ok = true, first = true;
    float acc_b3 = 0.f;
    double loss = 0.0;
    // the operand tiles written by every thread go to the tensor core
    auto publish = [&]() {
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
    };
    // every thread waits for the MMAs committed last; false (for all) if the wait ran out
    auto complete = [&]() -> bool {
        const bool done = mbar_wait(&S.mbar, phase, kWaitPolls);
        phase ^= 1u;
        tc_fence_after();
        return __syncthreads_and(done) != 0;
    };
    auto centred = [&](int br) -> float {
        const uint32_t code = group[perm[row0 + br]];
        const int q = (int)(code >> 16), size = (int)(code & 0xFFFFu);
        float mean = 0.f;
        for (int k = 0; k < size; ++k) mean += resid[br - q + k];
        return resid[br] - mean / (float)size;
    };
    // features and target of row r of tile `tile` (zero past the batch)
    auto load_x = [&](int tile, float (&x)[kNF], float& tg) {
        const int br = tile * kTcRows + r;
#pragma unroll
        for (int f = 0; f < kNF; ++f) x[f] = 0.f;
        tg = 0.f;
        if (br < B) {
            const int64_t src = perm[row0 + br];
            const float4 lo = *reinterpret_cast<const float4*>(feat + src * kNF);
            const float4 hi = *reinterpret_cast<const float4*>(feat + src * kNF + 4);
            x[0] = lo.x; x[1] = lo.y; x[2] = lo.z; x[3] = lo.w;
            x[4] = hi.x; x[5] = hi.y; x[6] = hi.z; x[7] = hi.w;
            tg = target[src];
        }
    };
    auto store_x = [&](int buf, const float (&x)[kNF]) {
        *reinterpret_cast<uint4*>(S.tX[buf] + blk_off(r, 0, kCX)) =
            make_uint4(pack_bf16(x[0], x[1]), pack_bf16(x[2], x[3]), pack_bf16(x[4], x[5]), pack_bf16(x[6], x[7]));
    };
    auto issue_g1 = [&](int buf) {
        umma_bf16(tmem + kD1, desc_kmajor(aX0 + (uint32_t)buf * (uint32_t)sizeof(S.tX[0]), kCX, 0),
                  desc_kmajor(aW1, kCX, 0), id64, false);
    };
    const int iters = (B + kTcRows - 1) / kTcRows;
    int it = blockIdx.x, buf = 0;
    float x[kNF], tg;
    load_x(it, x, tg);
    store_x(0, x);
    publish();
    if (tid == 0) {  // G1 of the first tile
        tc_fence_after();
        issue_g1(0);
        umma_commit(&S.mbar);
    }
    float gd1[kNH];  // gelu'(z1) of row r, from epilogue 1 to epilogue 3
    for (; it < iters; it += gridDim.x, buf ^= 1) {
        const int br = it * kTcRows + r;
        const bool valid = br < B;
        const int nxt = it + (int)gridDim.x;
        const bool has_next = nxt < iters;
        float xn[kNF], tgn;
        load_x(nxt, xn, tgn);  // in flight during this tile (zero if none)
        if (!(ok = complete())) break;  // G1 of this tile (and G5 of the previous one)
        // h1 = gelu(D1 + b1), and gelu'(z1) for the backward pass
#pragma unroll
        for (int c0 = 0; c0 < kNH; c0 += 16) {
            float d[16];
            tmem_ld16(tl + kD1 + c0, d);
            uint32_t p[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float h0, h1v;
                gelu_fd(d[2 * q] + S.b1[c0 + 2 * q], h0, gd1[c0 + 2 * q]);
                gelu_fd(d[2 * q + 1] + S.b1[c0 + 2 * q + 1], h1v, gd1[c0 + 2 * q + 1]);
                p[q] = pack_bf16(h0, h1v);
            }
            st_row16(S.tH, r, c0, kCH, p);
        }
        publish();
        if (tid == 0) {  // G2
            tc_fence_after();
#pragma unroll
            for (int k0 = 0; k0 < kNH; k0 += 16)
                umma_bf16(tmem + kD2, desc_kmajor(aH, kCH, k0), desc_kmajor(aW2, kNH, k0), id64, k0 > 0);
            umma_commit(&S.mbar);
        }
        if (!(ok = complete())) break;
        // h2 = gelu(D2 + b2) and the output y (bf16 h2, as the network's inference has it)
        float y = S.b3, gd2[kNH];
#pragma unroll
        for (int c0 = 0; c0 < kNH; c0 += 16) {
            float d[16];
            tmem_ld16(tl + kD2 + c0, d);
            uint32_t p[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float h0, h1v;
                gelu_fd(d[2 * q] + S.b2[c0 + 2 * q], h0, gd2[c0 + 2 * q]);
                gelu_fd(d[2 * q + 1] + S.b2[c0 + 2 * q + 1], h1v, gd2[c0 + 2 * q + 1]);
                p[q] = pack_bf16(h0, h1v);
                y = fmaf(bf16lo(p[q]), S.w3[c0 + 2 * q], y);
                y = fmaf(bf16hi(p[q]), S.w3[c0 + 2 * q + 1], y);
            }
            st_row16(S.tA, r, kNH + c0, kCA, p);
        }
        // dL/dy = 2 e / B, e the (centred) residual
        float dy = 0.f;
        if (valid) {
            const float e = resid ? centred(br) : y - tg;
            dy = 2.f * e * inv_b;
            loss += (double)e * e * inv_b;
        }
        acc_b3 += dy;
        // dz2 = dy w3 gelu'(z2)
#pragma unroll
        for (int c0 = 0; c0 < kNH; c0 += 16) {
            uint32_t p[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = c0 + 2 * q;
                p[q] = pack_bf16(dy * S.w3[c] * gd2[c], dy * S.w3[c + 1] * gd2[c + 1]);
            }
            st_row16(S.tA, r, c0, kCA, p);
        }
        {  // [1, dy_hi, dy_lo, 0 ...] beside h1
            const float dy_hi = __bfloat162float(__float2bfloat16_rn(dy));
            *reinterpret_cast<uint4*>(S.tH + blk_off(r, kNH, kCH)) =
                make_uint4(pack_bf16(1.f, dy_hi), pack_bf16(dy - dy_hi, 0.f), 0u, 0u);
        }
        publish();
        if (tid == 0) {  // G3 (into D2's columns, consumed) and G4
            tc_fence_after();
#pragma unroll
            for (int k0 = 0; k0 < kNH; k0 += 16)
                umma_bf16(tmem + kD2, desc_kmajor(aA, kCA, k0), desc_mnmajor(aW2, kNH, k0, 0), id3, k0 > 0);
#pragma unroll
            for (int k0 = 0; k0 < kTcRows; k0 += 16)
                umma_bf16(tmem + kD4, desc_mnmajor(aA, kCA, k0, 0), desc_mnmajor(aH, kCH, k0, 0), id4,
                          !first || k0 > 0);
            umma_commit(&S.mbar);
        }
        if (!(ok = complete())) break;
        // dz1 = dh1 gelu'(z1)
#pragma unroll
        for (int c0 = 0; c0 < kNH; c0 += 16) {
            float d[16];
            tmem_ld16(tl + kD2 + c0, d);
            uint32_t p[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int c = c0 + 2 * q;
                p[q] = pack_bf16(d[2 * q] * gd1[c], d[2 * q + 1] * gd1[c + 1]);
            }
            st_row16(S.tB, r, c0, kCB, p);
        }
        if (has_next) store_x(buf ^ 1, xn);
        publish();
        if (tid == 0) {  // G5 of this tile, G1 of the next
            tc_fence_after();
            const uint32_t aX = aX0 + (uint32_t)buf * (uint32_t)sizeof(S.tX[0]);
#pragma unroll
            for (int k0 = 0; k0 < kTcRows; k0 += 16)
                umma_bf16(tmem + kD5, desc_mnmajor(aB, kCB, k0, 0), desc_mnmajor(aX, kCX, k0, 0), id5,
                          !first || k0 > 0);
            if (has_next) issue_g1(buf ^ 1);
            umma_commit(&S.mbar);
        }
        first = false;
#pragma unroll
        for (int f = 0; f < kNF; ++f) x[f] = xn[f];
        tg = tgn;
    }
    if (ok && !first) ok = complete();  // the last G5
    // this CTA's partial sums: the weight and bias entries from TMEM (one
    // row per thread), b3 and the loss added in warp order
    float* prow = part + (size_t)blockIdx.x * kNParam;
    if (ok && !first) {
        float w3s = 0.f;
#pragma unroll 1
        for (int c0 = 0; c0 < 80; c0 += 16) {
            float d[16];
            tmem_ld16(tl + kD4 + c0, d);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int c = c0 + q;
                if (r < kNH) {
                    if (c < kNH) prow[oW2 + r * kNH + c] = d[q];
                    else if (c == kNH) prow[oB2 + r] = d[q];
                } else if (c == kNH + 1 || c == kNH + 2) {
                    w3s += d[q];
                }
            }
        }
        if (r >= kNH) prow[oW3 + r - kNH] = w3s;
        float d[16];
        tmem_ld16(tl + kD5, d);
        if (r < kNH) {
#pragma unroll
            for (int f = 0; f < kNF; ++f) prow[oW1 + r * kNF + f] = d[f];
            prow[oB1 + r] = d[kNF];
        }
    }
    for (int o = 16; o; o >>= 1) {
        acc_b3 += __shfl_xor_sync(kFull, acc_b3, o);
        loss += __shfl_xor_sync(kFull, loss, o);
    }
    if (lane == 0) {
        S.red[warp] = acc_b3;
        S.lred[warp] = loss;
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        float b3 = 0.f;
        double l = 0.0;
        for (int q = 0; q < kTcRows / 32; ++q) {
            b3 += S.red[q];
            l += S.lred[q];
        }
        prow[oB3] = b3;
        loss_part[blockIdx.x] = l;
        if (!ok) atomicExch(err, 1);
    }
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
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

// workspace: [0, 256) the device error word (int, zeroed by the caller), then
// the per-CTA partial sums and losses
size_t mlp_grad_workspace_bytes(int sm_count)
{
    return 256 + (size_t)2 * sm_count * (kNParam * sizeof(float) + sizeof(double)) + 256;
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
    const int smem = (int)sizeof(TcSmem);
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int iters = (B + kTcRows - 1) / kTcRows;
    const int grid = iters < 2 * sm_count ? iters : 2 * sm_count;  // two CTAs per SM (TMEM 2 x 256 columns)
    int* err = reinterpret_cast<int*>(work);
    float* part = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(work) + 256);
    double* loss_part = reinterpret_cast<double*>(
        reinterpret_cast<uint8_t*>(work) + 256 + ((size_t)2 * sm_count * kNParam * sizeof(float) + 255) / 256 * 256);
    mlp_grad_kernel<<<grid, kTcRows, smem, st>>>(M, feat, target, perm, row0, B, 1.0f / (float)B,
                                                 group ? resid : nullptr, group, part, loss_part, err);
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
