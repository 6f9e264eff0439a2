// pm_kernels.cu -- sm_103a kernels of the sparse-permanent estimator.
//
//  prepare_kernel      one CTA per matrix: validate A, build its CSC view,
//                      InitialDM (Sec. 2 / Alg. 2 preprocessing), compact to
//                      B0, K0 outer SK iterations (Sec. 3.3), initial degrees
//                      and minimum-degree tree.
//  (the trajectory kernel lives in pm_traj.cu)
//  stats kernels       ln mean X, p_match, relative spread, RSE, ESS (Sec. 2,
//                      Sec. 4 "Metrics").
#include <cmath>
#include <cstdio>
#include "pm_device.cuh"
#include "pm_dm.cuh"

namespace pm {

enum { VR_MD2 = 0, VR_ROW = 1 };
enum { SKP_NONE = 0, SKP_FIXED = 1, SKP_ADAPTIVE = 2, SKP_LOCAL = 3 };
enum { DMP_NONE = 0, DMP_ALL = 1, DMP_THRS = 2, DMP_TRCK = 3 };

// ---------------------------------------------------------------------------
// block helpers
// ---------------------------------------------------------------------------

// in-place inclusive scan of a[0..len) by one CTA
__device__ void block_inclusive_scan(int* a, int len)
{
    __shared__ int wsum[32];
    __shared__ int carry_s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    if (tid == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < len; base += blockDim.x) {
        const int i = base + tid;
        int v = i < len ? a[i] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) wsum[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int s = lane < nw ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, s, o);
                if (lane >= o) s += t;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        const int carry = carry_s;
        if (i < len) a[i] = v + (wid ? wsum[wid - 1] : 0) + carry;
        __syncthreads();
        if (tid == 0) carry_s = carry + wsum[nw - 1];
        __syncthreads();
    }
}

struct LiveAll {
    __device__ bool row(int) const { return true; }
    __device__ bool col(int) const { return true; }
    __device__ bool edge(int, int, int) const { return true; }
};

// ---------------------------------------------------------------------------
// preprocessing: one CTA per matrix
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(1024) prepare_kernel(DevMatrix* mats, const DevInput* inputs,
                                                       Sched s, uint32_t* status, int dyn_smem)
{
    DevMatrix& M = mats[blockIdx.x];
    const DevInput I = inputs[blockIdx.x];
    const int n = I.n, m = I.m, tid = threadIdx.x, nt = blockDim.x;
    __shared__ int bad_s, ok_s, unit_s;
    if (tid == 0) { bad_s = 0; ok_s = 1; unit_s = (I.val_in == nullptr); }
    __syncthreads();

    // 1. validate and copy A with int32 offsets
    for (int i = tid; i <= n; i += nt) {
        const int64_t p = I.rp64[i];
        if (p < 0 || p > m || (i == 0 && p != 0) || (i == n && p != m)) bad_s = 1;
        if (i < n && I.rp64[i + 1] < p) bad_s = 1;
        M.a_rp[i] = (int)p;
    }
    for (int e = tid; e < m; e += nt) {
        const int j = I.ci_in[e];
        if (j < 0 || j >= n) bad_s = 1;
        M.a_ci[e] = j;
        if (I.val_in) {
            const float v = I.val_in[e];
            if (!(v > 0.0f) || !(v <= 3.4028235e38f)) bad_s = 1;
            M.a_val[e] = v;
        }
    }
    __syncthreads();
    if (!bad_s) {
        for (int i = tid; i < n; i += nt)
            for (int e = M.a_rp[i] + 1; e < M.a_rp[i + 1]; ++e)
                if (M.a_ci[e] <= M.a_ci[e - 1]) bad_s = 1;
    }
    __syncthreads();
    if (bad_s) {
        if (tid == 0) { atomicOr(status, ST_BAD_INPUT); M.ok = 0; M.m = 0; }
        return;
    }

    // 2. CSC view of A (rows increasing inside each column)
    int* cursor = M.dm_ws;
    for (int j = tid; j <= n; j += nt) M.a_cp[j] = 0;
    __syncthreads();
    for (int e = tid; e < m; e += nt) atomicAdd(&M.a_cp[M.a_ci[e] + 1], 1);
    __syncthreads();
    block_inclusive_scan(M.a_cp + 1, n);
    for (int j = tid; j < n; j += nt) cursor[j] = M.a_cp[j];
    __syncthreads();
    for (int i = tid; i < n; i += nt)
        for (int e = M.a_rp[i]; e < M.a_rp[i + 1]; ++e) {
            const int k = atomicAdd(&cursor[M.a_ci[e]], 1);
            M.a_ri[k] = i;
            M.a_ce[k] = e;
        }
    __syncthreads();
    for (int j = tid; j < n; j += nt) {  // insertion sort of each column by row
        const int b = M.a_cp[j], en = M.a_cp[j + 1];
        for (int k = b + 1; k < en; ++k) {
            const int ri = M.a_ri[k], ce = M.a_ce[k];
            int q = k - 1;
            while (q >= b && M.a_ri[q] > ri) { M.a_ri[q + 1] = M.a_ri[q]; M.a_ce[q + 1] = M.a_ce[q]; --q; }
            M.a_ri[q + 1] = ri;
            M.a_ce[q + 1] = ce;
        }
    }
    for (int e = tid; e < m; e += nt) M.keep[e] = 1;
    __syncthreads();

    // 3. InitialDM (Alg. 2 preprocessing, Sec. 2); its workspace sits in shared
    // memory when the launch reserved enough (warp 0 runs it)
    extern __shared__ __align__(16) int dm_smem[];
    int* dm_ws = (dm_ws_ints(n) * 4 <= dyn_smem) ? dm_smem : M.dm_ws;
    if (s.initial_dm && n < 65536 && prep_stage_bytes(n, m) <= (size_t)dyn_smem) {
        // the search chases indices: stage A's adjacency in shared memory too
        // (the whole CTA copies, warp 0 searches)
        uint8_t* base = reinterpret_cast<uint8_t*>(dm_smem);
        size_t off = ((size_t)dm_ws_ints(n) * 4 + 15) / 16 * 16;
        int* s_rp = reinterpret_cast<int*>(base + off);
        off += ((size_t)(n + 1) * 4 + 15) / 16 * 16;
        int* s_cp = reinterpret_cast<int*>(base + off);
        off += ((size_t)(n + 1) * 4 + 15) / 16 * 16;
        uint16_t* s_ci = reinterpret_cast<uint16_t*>(base + off);
        off += ((size_t)m * 2 + 15) / 16 * 16;
        uint16_t* s_ri = reinterpret_cast<uint16_t*>(base + off);
        for (int i = tid; i <= n; i += nt) { s_rp[i] = M.a_rp[i]; s_cp[i] = M.a_cp[i]; }
        for (int e = tid; e < m; e += nt) { s_ci[e] = (uint16_t)M.a_ci[e]; s_ri[e] = (uint16_t)M.a_ri[e]; }
        __syncthreads();
        if (tid < 32) {
            const bool r = dm_warp(n, s_rp, s_ci, s_cp, s_ri, M.a_ce, LiveAll{}, M.keep, dm_smem, tid);
            if (tid == 0) ok_s = r ? 1 : 0;
        }
    } else if (s.initial_dm && tid < 32) {
        const bool r = dm_warp(n, M.a_rp, M.a_ci, M.a_cp, M.a_ri, M.a_ce, LiveAll{}, M.keep, dm_ws, tid);
        if (tid == 0) ok_s = r ? 1 : 0;
    }
    __syncthreads();
    const int ok = ok_s;
    // keep the initial DM's perfect matching (its edges are supported, so it
    // is one of B0): a trajectory's first inner DM repairs it instead of
    // matching from scratch
    if (s.initial_dm && ok) {
        const int* src = (s.initial_dm && n < 65536 && prep_stage_bytes(n, m) <= (size_t)dyn_smem) ? dm_smem : dm_ws;
        if (src != M.dm_ws)
            for (int q = tid; q < 2 * n; q += nt) M.dm_ws[q] = src[q];
    }
    if (tid == 0) M.matched = (s.initial_dm && ok) ? 1 : 0;

    // 4. compact to B0 (CSR, then CSC through the CSC view of A)
    for (int i = tid; i < n; i += nt) {
        int c = 0;
        for (int e = M.a_rp[i]; e < M.a_rp[i + 1]; ++e) c += M.keep[e];
        M.rp[i + 1] = c;
    }
    if (tid == 0) M.rp[0] = 0;
    __syncthreads();
    block_inclusive_scan(M.rp + 1, n);
    for (int i = tid; i < n; i += nt) {
        int q = M.rp[i];
        for (int e = M.a_rp[i]; e < M.a_rp[i + 1]; ++e) {
            if (!M.keep[e]) continue;
            M.ci[q] = M.a_ci[e];
            if (M.rv) M.rv[q] = M.a_val[e];
            ++q;
        }
    }
    for (int j = tid; j < n; j += nt) {
        int c = 0;
        for (int k = M.a_cp[j]; k < M.a_cp[j + 1]; ++k) c += M.keep[M.a_ce[k]];
        M.cp[j + 1] = c;
    }
    if (tid == 0) M.cp[0] = 0;
    __syncthreads();
    block_inclusive_scan(M.cp + 1, n);
    for (int j = tid; j < n; j += nt) {
        int q = M.cp[j];
        for (int k = M.a_cp[j]; k < M.a_cp[j + 1]; ++k) {
            const int e = M.a_ce[k];
            if (!M.keep[e]) continue;
            const int i = M.a_ri[k];
            // B0 id of A's edge e: position of e among the kept entries of row i
            int id = M.rp[i];
            for (int f = M.a_rp[i]; f < e; ++f) id += M.keep[f];
            M.ri[q] = i;
            M.ce[q] = id;
            if (M.cv) M.cv[q] = M.a_val[e];
            ++q;
        }
    }
    __syncthreads();

    // 5. outer scaling: K0 SK iterations on B0 from r = c = 1 (Sec. 3.3)
    Real* r0 = (Real*)M.r0;
    Real* c0 = (Real*)M.c0;
    for (int v = tid; v < n; v += nt) { r0[v] = (Real)1; c0[v] = (Real)1; }
    __syncthreads();
    const int K0 = ok ? s.K0 : 0;
    for (int it = 0; it < K0; ++it) {
        for (int j = tid; j < n; j += nt) {
            if (M.cp[j + 1] == M.cp[j]) continue;
            Real sum = 0;
            for (int k = M.cp[j]; k < M.cp[j + 1]; ++k) {
                const Real t = M.cv ? RA<Real>::mul((Real)M.cv[k], r0[M.ri[k]]) : r0[M.ri[k]];
                sum = RA<Real>::add(sum, t);
            }
            c0[j] = RA<Real>::rcp(sum);
        }
        __syncthreads();
        for (int i = tid; i < n; i += nt) {
            if (M.rp[i + 1] == M.rp[i]) continue;
            Real sum = 0;
            for (int e = M.rp[i]; e < M.rp[i + 1]; ++e) {
                const Real t = M.rv ? RA<Real>::mul((Real)M.rv[e], c0[M.ci[e]]) : c0[M.ci[e]];
                sum = RA<Real>::add(sum, t);
            }
            r0[i] = RA<Real>::rcp(sum);
        }
        __syncthreads();
    }
    for (int v = tid; v < n; v += nt)
        if (r0[v] != (Real)1 || c0[v] != (Real)1) unit_s = 0;

    // 6. initial degrees and minimum-degree tree
    const TreeGeom G = tree_geom(n);
    const int n2pad = (2 * n + 7) & ~7;
    for (int x = tid; x < n2pad; x += nt) {
        int d = kInact;
        if (x < n) d = M.rp[x + 1] - M.rp[x];
        else if (x < 2 * n) d = M.cp[x - n + 1] - M.cp[x - n];
        if (x < 2 * n && d > kMaxDegree) {  // live degrees are uint16
            atomicOr(status, ST_CAPACITY);
            d = kMaxDegree;
        }
        M.deg0[x] = (uint16_t)d;
    }
    __syncthreads();
    for (int l = 1; l <= G.nlev; ++l) {
        for (int gi = tid; gi < G.size[l]; gi += nt) {
            uint32_t best = 0xFFFFFFFFu;
            for (int q = 0; q < 32; ++q) {
                const int c = gi * 32 + q;
                if (c >= G.size[l - 1]) break;
                const uint32_t key = (l == 1) ? leaf_key(M.deg0, c, G) : M.tree0[G.off[l - 1] + c];
                best = key < best ? key : best;
            }
            M.tree0[G.off[l] + gi] = best;
        }
        __syncthreads();
    }
    __syncthreads();
    if (tid == 0) {
        M.ok = ok;
        M.m = M.rp[n];
        M.unit_scale = unit_s;
    }
}

// ---------------------------------------------------------------------------
// trajectory kernel
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// statistics: per chunk partial sums, then a fixed-order merge per matrix
// ---------------------------------------------------------------------------

__device__ double block_reduce_sum(double v, double* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int q = 0; q < nw; ++q) s += sh[q];
    __syncthreads();
    if (threadIdx.x == 0) sh[0] = s;
    __syncthreads();
    const double out = sh[0];
    __syncthreads();
    return out;
}

__device__ double block_reduce_max(double v, double* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = -INFINITY;
        for (int q = 0; q < nw; ++q) s = fmax(s, sh[q]);
        sh[0] = s;
    }
    __syncthreads();
    const double out = sh[0];
    __syncthreads();
    return out;
}

__global__ void __launch_bounds__(256) stats_partial_kernel(const double* log_x, const uint64_t* prefix,
                                                            int chunks, StatsPartial* parts)
{
    __shared__ double sh[32];
    const int k = blockIdx.y, ch = blockIdx.x;
    const uint64_t b0 = prefix[k], b1 = prefix[k + 1], len = b1 - b0;
    const uint64_t lo = b0 + len * ch / chunks, hi = b0 + len * (ch + 1) / chunks;
    // ln X = NaN marks a trajectory that a stopped launch never started: it
    // is not part of the sample (dead trajectories are -inf and count)
    double mx = -INFINITY, alive = 0, ran = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double v = log_x[i];
        if (v == v) ran += 1;
        if (v > -INFINITY) { mx = fmax(mx, v); alive += 1; }
    }
    mx = block_reduce_max(mx, sh);
    alive = block_reduce_sum(alive, sh);
    ran = block_reduce_sum(ran, sh);
    double s1 = 0, s2 = 0;
    if (mx > -INFINITY) {
        for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const double v = log_x[i];
            const double y = v > -INFINITY ? exp(v - mx) : 0.0;
            s1 += y;
            s2 += y * y;
        }
    }
    s1 = block_reduce_sum(s1, sh);
    s2 = block_reduce_sum(s2, sh);
    double m2 = 0;
    if (mx > -INFINITY) {
        const double mean = s1 / ran;
        for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const double v = log_x[i];
            if (!(v == v)) continue;
            const double y = v > -INFINITY ? exp(v - mx) : 0.0;
            m2 += (y - mean) * (y - mean);
        }
    }
    m2 = block_reduce_sum(m2, sh);
    if (threadIdx.x == 0) {
        StatsPartial& p = parts[(size_t)k * chunks + ch];
        p.c = mx; p.s1 = s1; p.s2 = s2; p.m2 = m2;
        p.cnt = (unsigned long long)ran;
        p.alive = (unsigned long long)alive;
    }
}

__global__ void stats_merge_kernel(const StatsPartial* parts, int chunks, int count, StatsOut* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const StatsPartial* P = parts + (size_t)k * chunks;
    double c = -INFINITY;
    unsigned long long n = 0, alive = 0;
    for (int q = 0; q < chunks; ++q) { c = fmax(c, P[q].c); n += P[q].cnt; alive += P[q].alive; }
    StatsOut o;
    o.n = n;
    o.alive = alive;
    o.p_match = n ? (double)alive / (double)n : 0.0;
    if (alive == 0) {
        o.log_estimate = o.log_sum_x = o.log_sum_x2 = -INFINITY;
        o.ess = 0; o.rel_spread = NAN; o.rse = NAN;
        out[k] = o;
        return;
    }
    // Chan et al. pairwise merge of (count, mean, M2) in shifted units
    double s1 = 0, s2 = 0, mean = 0, m2 = 0, na = 0;
    for (int q = 0; q < chunks; ++q) {
        if (P[q].cnt == 0) continue;
        const double f = (P[q].c > -INFINITY) ? exp(P[q].c - c) : 0.0;
        const double nb = (double)P[q].cnt;
        const double b1 = P[q].s1 * f, b2 = P[q].s2 * f * f, bm2 = P[q].m2 * f * f;
        const double mb = b1 / nb;
        const double d = mb - mean;
        const double nt = na + nb;
        mean = mean + d * nb / nt;
        m2 = m2 + bm2 + d * d * na * nb / nt;
        na = nt;
        s1 += b1;
        s2 += b2;
    }
    const double M = (double)n;
    const double mu = s1 / M;
    o.log_estimate = c + log(mu);
    o.log_sum_x = c + log(s1);
    o.log_sum_x2 = 2.0 * c + log(s2);
    o.ess = s1 * s1 / s2;
    o.rel_spread = (n > 1) ? sqrt(m2 / (M - 1.0)) / mu : NAN;
    o.rse = o.rel_spread / sqrt(M);
    out[k] = o;
}

__global__ void philox_kernel(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                              uint32_t count, uint32_t* out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    uint32_t x0 = c0 + i, x1 = c1, x2 = c2, x3 = c3;
    philox10(x0, x1, x2, x3, k0, k1);
    out[4 * i + 0] = x0; out[4 * i + 1] = x1; out[4 * i + 2] = x2; out[4 * i + 3] = x3;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

cudaError_t launch_prepare(DevMatrix* d_mats, const DevInput* d_in, int count, Sched s, int64_t m_max, int n_max,
                           uint32_t* status, cudaStream_t st)
{
    // shared memory for the initial DM: workspace and staged adjacency when
    // they fit, else the workspace only, else none (global memory)
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int dyn = 0;
    if (s.initial_dm) {
        const size_t staged = prep_stage_bytes(n_max, m_max);
        if (staged <= (size_t)(optin - 4096)) dyn = (int)staged;
        else if (dm_ws_ints(n_max) * 4 <= optin - 4096) dyn = dm_ws_ints(n_max) * 4;
    }
    // the cap stays at the device maximum (captured graphs of other calls may
    // hold larger launches of this kernel): opt-in less the static shared memory
    cudaFuncAttributes fa{};
    const cudaError_t ea = s.precision == 1 ? cudaFuncGetAttributes(&fa, (const void*)prepare_kernel<double>)
                                            : cudaFuncGetAttributes(&fa, (const void*)prepare_kernel<float>);
    if (ea != cudaSuccess) return ea;
    int cap = optin - (int)fa.sharedSizeBytes;
    if (cap < dyn) cap = dyn;
    cudaError_t e;
    if (s.precision == 1) {
        e = cudaFuncSetAttribute(prepare_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
        if (e != cudaSuccess) return e;
        prepare_kernel<double><<<count, 1024, dyn, st>>>(d_mats, d_in, s, status, dyn);
    } else {
        e = cudaFuncSetAttribute(prepare_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
        if (e != cudaSuccess) return e;
        prepare_kernel<float><<<count, 1024, dyn, st>>>(d_mats, d_in, s, status, dyn);
    }
    return cudaGetLastError();
}

cudaError_t launch_stats(const double* log_x, const uint64_t*, const uint64_t* d_prefix, int count,
                         StatsPartial* partials, int chunks, StatsOut* out, cudaStream_t st)
{
    stats_partial_kernel<<<dim3(chunks, count), 256, 0, st>>>(log_x, d_prefix, chunks, partials);
    stats_merge_kernel<<<(count + 63) / 64, 64, 0, st>>>(partials, chunks, count, out);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t count, uint32_t* out, cudaStream_t st)
{
    philox_kernel<<<(count + 127) / 128, 128, 0, st>>>(ctr[0], ctr[1], ctr[2], ctr[3], key[0], key[1], count, out);
    return cudaGetLastError();
}

}  // namespace pm
