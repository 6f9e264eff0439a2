// pm_device.cuh -- device helpers: Philox4x32-10, exact bounded draws, warp
// reductions, and binary32/binary64 arithmetic with explicit rounding (no
// contraction into FMA, so results are fixed by IEEE 754 alone).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "pm_internal.h"

namespace pm {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint16_t kInact = 0xFFFFu;

// ---- bounds checks of the PM_DEBUG build ----
// A checked array view (Chk) tests every index against the array's length and
// every value it returns against the values the array may hold (an adjacency
// index below n, a pointer at most m).  A violation is counted in this
// translation unit's bounds word and the access is replaced by element 0 and
// value 0, so it stays inside the array; the host reads the word after the
// call and fails it with PM_EDEVICE.  Release builds use plain pointers;
// raw() hands an array to code that takes plain pointers (unchecked).
#ifdef PM_DEBUG
static __device__ unsigned int g_pm_bounds;
__device__ __forceinline__ void pm_bounds_hit() { atomicAdd(&g_pm_bounds, 1u); }
template <typename T>
struct Chk {
    const T* p;
    uint32_t len;   // valid indices [0, len)
    uint32_t vmax;  // valid values [0, vmax)
    __device__ __forceinline__ T operator[](long long i) const
    {
        if ((unsigned long long)i >= (unsigned long long)len) {
            pm_bounds_hit();
            i = 0;
        }
        T v = p[i];
        if ((unsigned long long)(long long)v >= (unsigned long long)vmax) {
            pm_bounds_hit();
            v = 0;
        }
        return v;
    }
};
template <typename T>
using ChkPtr = Chk<T>;
template <typename T>
__device__ __forceinline__ const T* raw(const Chk<T>& c) { return c.p; }
#define PM_CLAMP(x, lim)                                                               \
    do {                                                                               \
        if ((unsigned long long)(long long)(x) >= (unsigned long long)(lim)) {         \
            pm_bounds_hit();                                                           \
            (x) = 0;                                                                   \
        }                                                                              \
    } while (0)
#else
template <typename T>
using ChkPtr = const T*;
template <typename T>
__device__ __forceinline__ const T* raw(const T* p) { return p; }
#define PM_CLAMP(x, lim) \
    do {                 \
    } while (0)
#endif

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// multiply-xor bijection, key bumped by the Weyl constants between rounds.
__device__ __forceinline__ void philox10(uint32_t& x0, uint32_t& x1, uint32_t& x2, uint32_t& x3,
                                         uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        const uint32_t a_hi = __umulhi(0xD2511F53u, x0), a_lo = 0xD2511F53u * x0;
        const uint32_t b_hi = __umulhi(0xCD9E8D57u, x2), b_lo = 0xCD9E8D57u * x2;
        const uint32_t n0 = b_hi ^ x1 ^ k0;
        const uint32_t n2 = a_hi ^ x3 ^ k1;
        x0 = n0; x1 = b_lo; x2 = n2; x3 = a_lo;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// 64-bit draw number `a` of (trajectory, matrix, step).  Counter words:
// (traj bits 0..31, traj bits 32..47 | matrix << 16, step, a >> 1); key: the
// two halves of the seed; even a -> words (0,1), odd a -> words (2,3).
__device__ __forceinline__ uint64_t draw_u64(uint64_t seed, uint64_t traj, uint32_t matrix,
                                             uint32_t step, uint32_t a)
{
    uint32_t x0 = (uint32_t)traj, x1 = (uint32_t)((traj >> 32) & 0xFFFFu) | (matrix << 16);
    uint32_t x2 = step, x3 = a >> 1;
    philox10(x0, x1, x2, x3, (uint32_t)seed, (uint32_t)(seed >> 32));
    return (a & 1u) ? (((uint64_t)x2 << 32) | x3) : (((uint64_t)x0 << 32) | x1);
}

// Exact uniform integer in [0, W): keep the high word of u*W unless the low
// word falls below 2^64 mod W (Lemire 2019).  u0 is draw 0 of the step, drawn
// by the caller ahead of time.  A low word >= W is above 2^64 mod W (< W), so
// the 64-bit remainder is only computed in the rare case (probability below
// W / 2^64) where the low word is < W; the decisions are those of the plain
// rule.  Returns ~0 when every allowed attempt was rejected.
__device__ __forceinline__ uint64_t uniform_below(uint64_t W, uint64_t u0, uint64_t seed, uint64_t traj,
                                                  uint32_t matrix, uint32_t step)
{
    if (u0 * W >= W) return __umul64hi(u0, W);
    const uint64_t reject_below = (0ull - W) % W;
    if (u0 * W >= reject_below) return __umul64hi(u0, W);
    for (uint32_t a = 1; a < (uint32_t)kMaxRngAttempts; ++a) {
        const uint64_t u = draw_u64(seed, traj, matrix, step, a);
        if (u * W >= reject_below) return __umul64hi(u, W);
    }
    return ~0ull;
}

// ---- warp collectives ----
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// maximum of non-negative values (their IEEE bit patterns order as integers)
__device__ __forceinline__ float warp_max_nonneg(float v)
{
    return __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(v)));
}
__device__ __forceinline__ double warp_max_nonneg(double v)
{
    long long b = __double_as_longlong(v);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const long long t = __shfl_xor_sync(kFull, b, o);
        b = t > b ? t : b;
    }
    return __longlong_as_double(b);
}

// ---- arithmetic of the proposal / scaling precision ----
template <typename Real> struct RA;
template <> struct RA<float> {
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }
    static __device__ __forceinline__ float pow2(int k) { return __int_as_float((127 + k) << 23); }
    static __device__ __forceinline__ unsigned long long to_u64(float x) { return __float2ull_rz(x); }
    static __device__ __forceinline__ float ceil_(float x) { return ceilf(x); }
};
template <> struct RA<double> {
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }
    static __device__ __forceinline__ double pow2(int k) { return __longlong_as_double((1023ll + k) << 52); }
    static __device__ __forceinline__ unsigned long long to_u64(double x) { return __double2ull_rz(x); }
    static __device__ __forceinline__ double ceil_(double x) { return ceil(x); }
};

// Integer proposal weight of a candidate with score s when the largest score
// is smax: max(1, floor((s / smax) * 2^k)); a NaN ratio gives 1.
template <typename Real>
__device__ __forceinline__ uint64_t quant_weight(Real s, Real smax, int k)
{
    const Real x = RA<Real>::mul(RA<Real>::div(s, smax), RA<Real>::pow2(k));
    return (x >= (Real)1) ? (uint64_t)RA<Real>::to_u64(x) : 1ull;
}

// packed (degree, unified id) key of leaf x of the minimum-degree tree;
// inactive vertices get the largest key
__device__ __forceinline__ uint32_t leaf_key(const uint16_t* deg, int x, const TreeGeom& G)
{
    const uint32_t d = deg[x];
    if (d == kInact) return 0xFFFFFFFFu;
    return ((d < G.dcap ? d : G.dcap) << G.idb) | (uint32_t)x;
}

// bit length of a positive 32-bit value
__device__ __forceinline__ int bitlen(uint32_t x) { return 32 - __clz(x); }

// A positive number kept as m * 2^e with a 64-bit mantissa m in [2^63, 2^64):
// the running products of Algorithm 2's correction (prod W B and prod w)
// without floating-point units.  Multiplying by an integer keeps the top 64
// bits of the exact 128-bit product (truncation: relative error below 2^-63
// per product, finer than binary64).
struct Mant64 {
    uint64_t m = 1ull << 63;
    int e = -63;
    __device__ __forceinline__ void mul(uint64_t w)  // w >= 1
    {
        const uint64_t lo = m * w, hi = __umul64hi(m, w);
        if (hi == 0) return;  // w == 1
        const int lz = __clzll(hi);
        m = (hi << lz) | (lz ? (lo >> (64 - lz)) : 0ull);
        e += 64 - lz;
    }
    // multiply by a positive finite binary32 value, exactly its 24-bit
    // integer significand times a power of two
    __device__ __forceinline__ void mul(float x)
    {
        const uint32_t b = __float_as_uint(x);
        const uint32_t ef = (b >> 23) & 0xFFu;
        const uint32_t sig = ef ? ((b & 0x7FFFFFu) | 0x800000u) : (b & 0x7FFFFFu);
        mul((uint64_t)sig);
        e += (ef ? (int)ef : 1) - 127 - 23;
    }
    // ln of the value; explicit roundings (no contraction into an FMA), so
    // every kernel that inlines it produces the same bits
    __device__ __forceinline__ double log_value() const
    {
        return __dadd_rn(log((double)m), __dmul_rn((double)e, 0.6931471805599453));
    }
};

// ln(num / den) of two Mant64 accumulators
__device__ __forceinline__ double log_ratio(const Mant64& num, const Mant64& den)
{
    return __dsub_rn(num.log_value(), den.log_value());
}

}  // namespace pm
