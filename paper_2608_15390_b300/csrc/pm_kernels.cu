// pm_kernels.cu -- sm_103a kernels of the sparse-permanent estimator.
//
//  prepare_kernel      one CTA per matrix: validate A, build its CSC view,
//                      InitialDM (Sec. 2 / Alg. 2 preprocessing), compact to
//                      B0, K0 outer SK iterations (Sec. 3.3), initial degrees
//                      and minimum-degree tree.
//  traj_kernel         persistent; one warp per trajectory (Alg. 2): two-sided
//                      minimum-degree pick (Sec. 3.2), scaled proposal (Eq. 3),
//                      importance correction, elimination with degree updates,
//                      DM policy (Sec. 3.3), SK policy (Sec. 3.3, Eq. 5).
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

__device__ __forceinline__ uint32_t leaf_key(const uint16_t* deg, int x, const TreeGeom& G)
{
    const uint32_t d = deg[x];
    if (d == kInact) return 0xFFFFFFFFu;
    return ((d < G.dcap ? d : G.dcap) << G.idb) | (uint32_t)x;
}

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
                                                       Sched s, uint32_t* status)
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

    // 3. InitialDM (Alg. 2 preprocessing, Sec. 2)
    if (s.initial_dm && tid == 0)
        ok_s = dm_serial(n, M.a_rp, M.a_ci, M.a_cp, M.a_ri, M.a_ce, LiveAll{}, M.keep, M.dm_ws) ? 1 : 0;
    __syncthreads();
    const int ok = ok_s;

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
        uint16_t d = kInact;
        if (x < n) d = (uint16_t)(M.rp[x + 1] - M.rp[x]);
        else if (x < 2 * n) d = (uint16_t)(M.cp[x - n + 1] - M.cp[x - n]);
        M.deg0[x] = d;
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

struct LiveTraj {
    const uint16_t* deg;
    const uint8_t* mask;
    int n;
    __device__ bool row(int i) const { return deg[i] != kInact; }
    __device__ bool col(int j) const { return deg[n + j] != kInact; }
    __device__ bool edge(int e, int i, int j) const
    {
        return mask[e] && deg[i] != kInact && deg[n + j] != kInact;
    }
};

// lower the tree entries above leaf x to (at most) its new key
__device__ __forceinline__ void tree_lower(uint32_t* tree, const TreeGeom& G, int x, uint32_t d)
{
    const uint32_t key = ((d < G.dcap ? d : G.dcap) << G.idb) | (uint32_t)x;
    for (int l = 1; l <= G.nlev; ++l) atomicMin(&tree[G.off[l] + (x >> (5 * l))], key);
}

// recompute the tree entries above leaves x and y from their children
__device__ void tree_fix2(const uint16_t* deg, uint32_t* tree, const TreeGeom& G, int x, int y, int lane)
{
    for (int l = 1; l <= G.nlev; ++l) {
        const int gx = x >> (5 * l), gy = y >> (5 * l);
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            const int gi = w ? gy : gx;
            if (w && gy == gx) break;
            const int c = gi * 32 + lane;
            uint32_t key = 0xFFFFFFFFu;
            if (c < G.size[l - 1]) key = (l == 1) ? leaf_key(deg, c, G) : tree[G.off[l - 1] + c];
            key = __reduce_min_sync(kFull, key);
            if (lane == 0) tree[G.off[l] + gi] = key;
        }
        __syncwarp();
    }
}

__device__ void tree_build(const uint16_t* deg, uint32_t* tree, const TreeGeom& G, int lane)
{
    for (int l = 1; l <= G.nlev; ++l) {
        for (int gi = lane; gi < G.size[l]; gi += 32) {
            uint32_t best = 0xFFFFFFFFu;
            for (int q = 0; q < 32; ++q) {
                const int c = gi * 32 + q;
                if (c >= G.size[l - 1]) break;
                const uint32_t key = (l == 1) ? leaf_key(deg, c, G) : tree[G.off[l - 1] + c];
                best = key < best ? key : best;
            }
            tree[G.off[l] + gi] = best;
        }
        __syncwarp();
    }
}

// two-sided minimum degree: the active vertex of least (degree, unified id)
__device__ __forceinline__ int md_pick(const uint16_t* deg, const uint32_t* tree, const TreeGeom& G,
                                       int lane)
{
    uint32_t key = 0xFFFFFFFFu;
    if (G.nlev == 0) {
        if (lane < G.n2) key = leaf_key(deg, lane, G);
    } else if (lane < G.size[G.nlev]) {
        key = tree[G.off[G.nlev] + lane];
    }
    key = __reduce_min_sync(kFull, key);
    if ((key >> G.idb) < G.dcap) return (int)(key & ((1u << G.idb) - 1u));
    // saturated degree field: exact scan with full degrees
    unsigned long long best = ~0ull;
    for (int x = lane; x < G.n2; x += 32) {
        const uint32_t d = deg[x];
        if (d == kInact) continue;
        const unsigned long long k64 = ((unsigned long long)d << 32) | (unsigned)x;
        best = k64 < best ? k64 : best;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(kFull, best, o);
        best = t < best ? t : best;
    }
    return (int)(best & 0xFFFFFFFFu);
}

struct MatView {
    int n;
    const int *rp, *ci, *cp, *ri, *ce;
    const float *rv, *cv;
};

// live edge test for position e of a row list (CSR, id e) or a column list
// (CSC, id ce[e]); partner unified id pid
__device__ __forceinline__ bool entry_live(const uint16_t* deg, const uint8_t* mask, const MatView& V,
                                           bool row_list, int e, int pid)
{
    if (deg[pid] == kInact) return false;
    if (!mask) return true;
    return mask[row_list ? e : __ldg(V.ce + e)] != 0;
}

// one SK iteration on the residual: every active column from r, then every
// active row from the new c; vertices without live edges keep their scale
template <typename Real>
__device__ void sk_sweep(const MatView& V, const uint16_t* deg, const uint8_t* mask, Real* r, Real* c,
                         int lane)
{
    const int n = V.n;
    for (int j = lane; j < n; j += 32) {
        const uint16_t dj = deg[n + j];
        if (dj == kInact || dj == 0) continue;
        Real sum = 0;
        const int b = __ldg(V.cp + j), en = __ldg(V.cp + j + 1);
        for (int k = b; k < en; ++k) {
            const int i = __ldg(V.ri + k);
            if (deg[i] == kInact || (mask && !mask[__ldg(V.ce + k)])) continue;
            const Real t = V.cv ? RA<Real>::mul((Real)__ldg(V.cv + k), r[i]) : r[i];
            sum = RA<Real>::add(sum, t);
        }
        c[j] = RA<Real>::rcp(sum);
    }
    __syncwarp();
    for (int i = lane; i < n; i += 32) {
        const uint16_t di = deg[i];
        if (di == kInact || di == 0) continue;
        Real sum = 0;
        const int b = __ldg(V.rp + i), en = __ldg(V.rp + i + 1);
        for (int e = b; e < en; ++e) {
            const int j = __ldg(V.ci + e);
            if (deg[n + j] == kInact || (mask && !mask[e])) continue;
            const Real t = V.rv ? RA<Real>::mul((Real)__ldg(V.rv + e), c[j]) : c[j];
            sum = RA<Real>::add(sum, t);
        }
        r[i] = RA<Real>::rcp(sum);
    }
    __syncwarp();
}

template <typename Real>
__device__ __forceinline__ Real row_scale_new(const MatView& V, const uint16_t* deg, const uint8_t* mask,
                                              const Real* r, const Real* c, int i)
{
    if (deg[i] == 0) return r[i];
    Real sum = 0;
    const int b = __ldg(V.rp + i), en = __ldg(V.rp + i + 1);
    for (int e = b; e < en; ++e) {
        const int j = __ldg(V.ci + e);
        if (deg[V.n + j] == kInact || (mask && !mask[e])) continue;
        const Real t = V.rv ? RA<Real>::mul((Real)__ldg(V.rv + e), c[j]) : c[j];
        sum = RA<Real>::add(sum, t);
    }
    return RA<Real>::rcp(sum);
}

template <typename Real>
__device__ __forceinline__ Real col_scale_new(const MatView& V, const uint16_t* deg, const uint8_t* mask,
                                              const Real* r, const Real* c, int j)
{
    if (deg[V.n + j] == 0) return c[j];
    Real sum = 0;
    const int b = __ldg(V.cp + j), en = __ldg(V.cp + j + 1);
    for (int k = b; k < en; ++k) {
        const int i = __ldg(V.ri + k);
        if (deg[i] == kInact || (mask && !mask[__ldg(V.ce + k)])) continue;
        const Real t = V.cv ? RA<Real>::mul((Real)__ldg(V.cv + k), r[i]) : r[i];
        sum = RA<Real>::add(sum, t);
    }
    return RA<Real>::rcp(sum);
}

// Local repair (Eq. 5).  lr[0..nr): N_t(C)\{R} (rows); lc[0..nc): N_t(R)\{C}
// (columns).  R_loc = lr U N_{t+1}(lc), C_loc = lc U N_{t+1}(lr).  New rows
// are staged (deduplicated by stamp) because they read the old c; columns
// then read the old r and are written in place; the staged rows commit last.
template <typename Real>
__device__ void local_repair(const MatView& V, const uint16_t* deg, const uint8_t* mask, Real* r, Real* c,
                             const int* lr, int nr, const int* lc, int nc, int* stamp, int st,
                             int* tmp_id, Real* tmp_val, int* tmp_cnt, int lane)
{
    const int n = V.n;
    if (lane == 0) *tmp_cnt = 0;
    __syncwarp();
    auto stage_row = [&](int i) {
        if (atomicExch(&stamp[i], st) == st) return;
        const Real v = row_scale_new<Real>(V, deg, mask, r, c, i);
        const int q = atomicAdd(tmp_cnt, 1);
        tmp_id[q] = i;
        tmp_val[q] = v;
    };
    for (int q = lane; q < nr; q += 32) stage_row(lr[q]);
    for (int q = lane; q < nc; q += 32) {
        const int j = lc[q];
        const int b = __ldg(V.cp + j), en = __ldg(V.cp + j + 1);
        for (int k = b; k < en; ++k) {
            const int i = __ldg(V.ri + k);
            if (deg[i] == kInact || (mask && !mask[__ldg(V.ce + k)])) continue;
            stage_row(i);
        }
    }
    __syncwarp();
    // columns: values depend only on the old r, duplicates write equal values
    for (int q = lane; q < nc; q += 32) {
        const int j = lc[q];
        c[j] = col_scale_new<Real>(V, deg, mask, r, c, j);
    }
    for (int q = lane; q < nr; q += 32) {
        const int i = lr[q];
        const int b = __ldg(V.rp + i), en = __ldg(V.rp + i + 1);
        for (int e = b; e < en; ++e) {
            const int j = __ldg(V.ci + e);
            if (deg[n + j] == kInact || (mask && !mask[e])) continue;
            c[j] = col_scale_new<Real>(V, deg, mask, r, c, j);
        }
    }
    __syncwarp();
    const int cnt = *tmp_cnt;
    for (int q = lane; q < cnt; q += 32) r[tmp_id[q]] = tmp_val[q];
    __syncwarp();
}

template <typename Real>
__device__ __forceinline__ Real cand_score(const MatView& V, bool vrow, int e, int p, const Real* r,
                                           const Real* c)
{
    const float* vals = vrow ? V.rv : V.cv;
    const Real sc = vrow ? c[p] : r[p];
    Real s = vals ? RA<Real>::mul((Real)__ldg(vals + e), sc) : sc;
    if (!(s >= (Real)0)) s = 0;
    return s;
}

template <typename Real, bool TRACE>
__device__ void run_trajectory(const TrajParams& P, int k, uint64_t g, uint64_t local, uint16_t* deg,
                               uint32_t* tree, int* misc, uint8_t* slot, int lane)
{
    const DevMatrix* Mp = P.mats + k;
    const int n = Mp->n;
    const int ok = Mp->ok;
    const uint64_t traj = P.first_traj + local;
    const uint32_t midx = (uint32_t)Mp->idx;
    const Sched& S = P.s;
    if (TRACE) {
        for (int q = lane; q < 2 * n; q += 32) P.chosen[g * 2 * n + q] = -1;
        for (int q = lane; q < n; q += 32) P.deg_v[g * n + q] = -1;
    }
    if (!ok) {
        if (lane == 0) {
            P.log_x[g] = -INFINITY;
            if (TRACE) P.dead_step[g] = 0;
        }
        return;
    }
    MatView V;
    V.n = n;
    V.rp = Mp->rp; V.ci = Mp->ci; V.cp = Mp->cp; V.ri = Mp->ri; V.ce = Mp->ce;
    V.rv = Mp->rv; V.cv = Mp->cv;
    const TreeGeom G = tree_geom(n);

    // trajectory state from the shared initial state
    {
        const uint4* src = reinterpret_cast<const uint4*>(Mp->deg0);
        uint4* dst = reinterpret_cast<uint4*>(deg);
        const int nv = (2 * n + 7) / 8;
        for (int q = lane; q < nv; q += 32) dst[q] = __ldg(src + q);
        for (int q = lane; q < G.total; q += 32) tree[q] = __ldg(Mp->tree0 + q);
    }
    const bool inner_sk = S.sk != SKP_NONE;
    const bool use_dm = S.dm != DMP_NONE;
    const bool use_local = S.sk == SKP_LOCAL;
    Real* r;
    Real* c;
    if (inner_sk) {
        r = reinterpret_cast<Real*>(slot + P.slot.r);
        c = reinterpret_cast<Real*>(slot + P.slot.c);
        const Real* r0 = reinterpret_cast<const Real*>(Mp->r0);
        const Real* c0 = reinterpret_cast<const Real*>(Mp->c0);
        for (int q = lane; q < n; q += 32) { r[q] = r0[q]; c[q] = c0[q]; }
    } else {
        r = reinterpret_cast<Real*>(Mp->r0);
        c = reinterpret_cast<Real*>(Mp->c0);
    }
    uint8_t* mask = nullptr;
    int* dmws = nullptr;
    if (use_dm) {
        mask = slot + P.slot.mask;
        dmws = reinterpret_cast<int*>(slot + P.slot.dm);
        const int m = Mp->m;
        for (int q = lane; q < m; q += 32) mask[q] = 1;
    }
    int *stamp = nullptr, *tmp_id = nullptr, *list_r = nullptr, *list_c = nullptr;
    Real* tmp_val = nullptr;
    if (use_local) {
        stamp = reinterpret_cast<int*>(slot + P.slot.stamp);
        tmp_id = reinterpret_cast<int*>(slot + P.slot.tmp_id);
        tmp_val = reinterpret_cast<Real*>(slot + P.slot.tmp_val);
        list_r = reinterpret_cast<int*>(slot + P.slot.list_r);
        list_c = reinterpret_cast<int*>(slot + P.slot.list_c);
        for (int q = lane; q < n; q += 32) stamp[q] = 0;
    }
    __syncwarp();

    const bool uniform = Mp->unit_scale && !inner_sk;
    const Real theta = (Real)S.theta;
    double num = 1.0, den = 1.0;  // X = num / den * 2^ex (lane 0)
    int ex = 0;
    Real track = 1;
    unsigned n_dm = 0, n_full = 0, n_loc = 0;
    int dead_step = -1;
    // algorithmic bytes (lane 0): per step 8 B per adjacency entry of the
    // picked vertex and its partner (index + state), per full SK iteration
    // 16 B per live edge, per Local repair 16 B per staged vertex and
    // neighbour; m_live = live edges of the residual
    uint64_t alg_bytes = (uint64_t)2 * n * 4;
    int m_live = Mp->m;

    for (int t = 0; t < n; ++t) {
        const int v = (S.vertex_rule == VR_ROW) ? t : md_pick(deg, tree, G, lane);
        const int dv = deg[v];
        if (TRACE && lane == 0) P.deg_v[g * n + t] = dv;
        if (dv == 0) { dead_step = t; break; }

        const bool vrow = v < n;
        const int vi = vrow ? v : v - n;
        const int beg = __ldg((vrow ? V.rp : V.cp) + vi);
        const int end = __ldg((vrow ? V.rp : V.cp) + vi + 1);
        const int* adj = vrow ? V.ci : V.ri;
        const int poff = vrow ? n : 0;
        const int kq = 40 - bitlen((uint32_t)dv);
        const int len = end - beg;

        uint64_t W = 0, w_sel = 0;
        int sel_e = -1, sel_p = -1;
        bool keep_live = false;
        int keep_pid = 0;
        uint64_t rr;
        if (len <= 32) {
            const int e = beg + lane;
            const bool in = lane < len;
            const int pp = in ? __ldg(adj + e) : 0;
            const bool live = in && entry_live(deg, mask, V, vrow, e, pp + poff);
            const unsigned lm = __ballot_sync(kFull, live);
            uint64_t w;
            if (uniform) {
                w = live ? (1ull << kq) : 0ull;
                W = (uint64_t)dv << kq;
            } else {
                const Real sv = live ? cand_score<Real>(V, vrow, e, pp, r, c) : (Real)0;
                const Real smax = warp_max_nonneg(sv);
                w = live ? quant_weight<Real>(sv, smax, kq) : 0ull;
                W = warp_sum_u64(w);
            }
            rr = uniform_below(W, P.seed, traj, midx, (uint32_t)t);
            if (rr == ~0ull) {
                if (lane == 0) atomicOr(P.status, ST_RNG_EXHAUSTED);
                dead_step = t;
                break;
            }
            int sl;
            if (uniform) {
                unsigned mm = lm;  // drop the first (rr >> kq) live lanes
                for (int q = (int)(rr >> kq); q > 0; --q) mm &= mm - 1u;
                sl = __ffs(mm) - 1;
            } else {
                const uint64_t pre = warp_incl_scan_u64(w, lane);
                const unsigned hit = __ballot_sync(kFull, live && pre > rr);
                sl = __ffs(hit) - 1;
            }
            if (sl >= 0) {
                sel_e = __shfl_sync(kFull, e, sl);
                sel_p = __shfl_sync(kFull, pp, sl);
                w_sel = __shfl_sync(kFull, w, sl);
            }
            keep_live = live && pp != sel_p;
            keep_pid = pp + poff;
        } else {
            Real smax = 0;
            if (!uniform) {
                for (int base = beg; base < end; base += 32) {
                    const int e = base + lane;
                    Real sv = 0;
                    if (e < end) {
                        const int pp = __ldg(adj + e);
                        if (entry_live(deg, mask, V, vrow, e, pp + poff)) sv = cand_score<Real>(V, vrow, e, pp, r, c);
                    }
                    const Real cm = warp_max_nonneg(sv);
                    smax = cm > smax ? cm : smax;
                }
                for (int base = beg; base < end; base += 32) {
                    const int e = base + lane;
                    uint64_t w = 0;
                    if (e < end) {
                        const int pp = __ldg(adj + e);
                        if (entry_live(deg, mask, V, vrow, e, pp + poff))
                            w = quant_weight<Real>(cand_score<Real>(V, vrow, e, pp, r, c), smax, kq);
                    }
                    W += warp_sum_u64(w);
                }
            } else {
                W = (uint64_t)dv << kq;
            }
            rr = uniform_below(W, P.seed, traj, midx, (uint32_t)t);
            if (rr == ~0ull) {
                if (lane == 0) atomicOr(P.status, ST_RNG_EXHAUSTED);
                dead_step = t;
                break;
            }
            uint64_t carry = 0;
            for (int base = beg; base < end; base += 32) {
                const int e = base + lane;
                int pp = 0;
                bool live = false;
                uint64_t w = 0;
                if (e < end) {
                    pp = __ldg(adj + e);
                    live = entry_live(deg, mask, V, vrow, e, pp + poff);
                    if (live) w = uniform ? (1ull << kq) : quant_weight<Real>(cand_score<Real>(V, vrow, e, pp, r, c), smax, kq);
                }
                const uint64_t pre = warp_incl_scan_u64(w, lane) + carry;
                const unsigned hit = __ballot_sync(kFull, live && pre > rr);
                if (hit) {
                    const int sl = __ffs(hit) - 1;
                    sel_e = __shfl_sync(kFull, e, sl);
                    sel_p = __shfl_sync(kFull, pp, sl);
                    w_sel = __shfl_sync(kFull, w, sl);
                    break;
                }
                carry = __shfl_sync(kFull, pre, 31);
            }
        }
        if (sel_p < 0 || sel_e < beg || sel_e >= end) {  // cannot happen unless degrees are corrupt
            if (lane == 0) atomicOr(P.status, ST_INTERNAL);
            dead_step = t;
            break;
        }
        const int u = sel_p + poff;               // unified id of the partner
        const int R = vrow ? vi : sel_p;          // matched row
        const int C = vrow ? sel_p : vi;          // matched column
        if (TRACE && lane == 0) {
            P.chosen[(g * n + t) * 2 + 0] = v;
            P.chosen[(g * n + t) * 2 + 1] = u;
        }
        // correction X <- X * B_vu * W / w_u
        if (lane == 0) {
            num = num * (double)W;
            const float* vals = vrow ? V.rv : V.cv;
            if (vals) num = num * (double)__ldg(vals + sel_e);
            den = den * (double)w_sel;
            ex += renorm(num);
            ex -= renorm(den);
        }
        const Real z = RA<Real>::mul(r[R], c[C]);

        // elimination of R and C, degree and tree updates
        __syncwarp();
        if (lane == 0) { deg[R] = kInact; deg[n + C] = kInact; }
        __syncwarp();
        int cnt_r = 0, cnt_c = 0;  // local-repair lists (warp-uniform counts)
        int* list_v = vrow ? list_c : list_r;
        int* list_u = vrow ? list_r : list_c;
        int cnt_v = 0, cnt_u = 0;
        if (len <= 32) {
            if (keep_live) {
                const uint32_t d = deg[keep_pid] - 1u;
                deg[keep_pid] = (uint16_t)d;
                tree_lower(tree, G, keep_pid, d);
            }
            if (use_local) {
                const unsigned km = __ballot_sync(kFull, keep_live);
                if (keep_live) list_v[__popc(km & ((1u << lane) - 1u))] = keep_pid - poff;
                cnt_v = __popc(km);
            }
        } else {
            for (int base = beg; base < end; base += 32) {
                const int e = base + lane;
                bool live = false;
                int pid = 0;
                if (e < end) {
                    pid = __ldg(adj + e) + poff;
                    live = entry_live(deg, mask, V, vrow, e, pid);
                }
                if (live) {
                    const uint32_t d = deg[pid] - 1u;
                    deg[pid] = (uint16_t)d;
                    tree_lower(tree, G, pid, d);
                }
                if (use_local) {
                    const unsigned km = __ballot_sync(kFull, live);
                    if (live) list_v[cnt_v + __popc(km & ((1u << lane) - 1u))] = pid - poff;
                    cnt_v += __popc(km);
                }
            }
        }
        int n_u_live = 0, ue_len = 0;
        {   // the partner's list
            const bool urow = !vrow;
            const int ui = sel_p;
            const int ub = __ldg((urow ? V.rp : V.cp) + ui);
            const int ue = __ldg((urow ? V.rp : V.cp) + ui + 1);
            const int* uadj = urow ? V.ci : V.ri;
            const int uoff = urow ? n : 0;
            ue_len = ue - ub;
            for (int base = ub; base < ue; base += 32) {
                const int e = base + lane;
                bool live = false;
                int pid = 0;
                if (e < ue) {
                    pid = __ldg(uadj + e) + uoff;
                    live = entry_live(deg, mask, V, urow, e, pid);
                }
                if (live) {
                    const uint32_t d = deg[pid] - 1u;
                    deg[pid] = (uint16_t)d;
                    tree_lower(tree, G, pid, d);
                }
                const unsigned km = __ballot_sync(kFull, live);
                if (use_local && live) list_u[cnt_u + __popc(km & ((1u << lane) - 1u))] = pid - uoff;
                cnt_u += __popc(km);
            }
            n_u_live = cnt_u;
        }
        cnt_r = vrow ? cnt_u : cnt_v;
        cnt_c = vrow ? cnt_v : cnt_u;
        m_live -= dv + n_u_live;
        alg_bytes += (uint64_t)8 * (uint64_t)(len + (ue_len));
        __syncwarp();
        if (S.vertex_rule != VR_ROW) tree_fix2(deg, tree, G, R, n + C, lane);
        (void)u;
        track = RA<Real>::mul(track, z);

        if (t + 1 < n) {
            const bool run_dm = (S.dm == DMP_ALL) || (S.dm == DMP_THRS && z < theta) ||
                                (S.dm == DMP_TRCK && track < theta);
            if (run_dm) {
                ++n_dm;
                int okdm = 0;
                if (lane == 0)
                    okdm = dm_serial(n, V.rp, V.ci, V.cp, V.ri, V.ce, LiveTraj{deg, mask, n}, mask, dmws) ? 1 : 0;
                okdm = __shfl_sync(kFull, okdm, 0);
                __syncwarp();
                if (!okdm) { dead_step = t; break; }
                // live degrees of the filtered child, then the tree
                for (int x = lane; x < 2 * n; x += 32) {
                    if (deg[x] == kInact) continue;
                    int d = 0;
                    if (x < n) {
                        for (int e = __ldg(V.rp + x); e < __ldg(V.rp + x + 1); ++e)
                            d += (mask[e] && deg[n + __ldg(V.ci + e)] != kInact);
                    } else {
                        const int j = x - n;
                        for (int kk = __ldg(V.cp + j); kk < __ldg(V.cp + j + 1); ++kk)
                            d += (mask[__ldg(V.ce + kk)] && deg[__ldg(V.ri + kk)] != kInact);
                    }
                    deg[x] = (uint16_t)d;
                }
                __syncwarp();
                tree_build(deg, tree, G, lane);
                track = 1;
                int ml = 0;  // live edges of the filtered child: sum of row degrees
                for (int x = lane; x < n; x += 32) ml += (deg[x] != kInact) ? deg[x] : 0;
#pragma unroll
                for (int o = 16; o; o >>= 1) ml += __shfl_xor_sync(kFull, ml, o);
                m_live = ml;
            }
            if (S.sk == SKP_FIXED || S.sk == SKP_ADAPTIVE) {
                int nit = S.K;
                if (S.sk == SKP_ADAPTIVE) {
                    const Real b = RA<Real>::mul(RA<Real>::sub((Real)1, z), (Real)S.K);
                    nit = (b > (Real)0) ? (int)RA<Real>::ceil_(b) : 0;
                }
                for (int q = 0; q < nit; ++q) sk_sweep<Real>(V, deg, mask, r, c, lane);
                n_full += nit;
                alg_bytes += (uint64_t)16 * (uint64_t)m_live * (uint64_t)nit;
            } else if (S.sk == SKP_LOCAL) {
                local_repair<Real>(V, deg, mask, r, c, list_r, cnt_r, list_c, cnt_c, stamp, t + 1, tmp_id,
                                   tmp_val, misc, lane);
                ++n_loc;
                alg_bytes += (uint64_t)16 * (uint64_t)(*misc + cnt_r + cnt_c);
            }
        }
    }
    if (lane == 0) {
        P.log_x[g] = (dead_step >= 0) ? -INFINITY : (log(num) - log(den)) + (double)ex * 0.6931471805599453;
        if (TRACE) P.dead_step[g] = dead_step;
        if (n_dm) atomicAdd(P.counters + 4 * k + 0, (unsigned long long)n_dm);
        if (n_full) atomicAdd(P.counters + 4 * k + 1, (unsigned long long)n_full);
        if (n_loc) atomicAdd(P.counters + 4 * k + 2, (unsigned long long)n_loc);
        atomicAdd(P.counters + 4 * k + 3, (unsigned long long)alg_bytes);
    }
    __syncwarp();
}

constexpr int kTrajWarpsPerCta = 8;

int traj_smem_per_warp(int n_max)
{
    const TreeGeom G = tree_geom(n_max);
    const int deg_bytes = (int)align_up((size_t)((2 * n_max + 7) & ~7) * 2, 16);
    const int tree_bytes = (int)align_up((size_t)G.total * 4, 16);
    return deg_bytes + tree_bytes + 16;
}

int traj_kernel_max_warps_per_cta() { return kTrajWarpsPerCta; }

template <typename Real, bool TRACE>
__global__ void __launch_bounds__(kTrajWarpsPerCta * 32) traj_kernel(TrajParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    uint8_t* base = smem + (size_t)wib * P.smem_per_warp;
    const TreeGeom Gmax = tree_geom(P.n_max);
    const int deg_bytes = (int)(((((2 * P.n_max + 7) & ~7) * 2) + 15) & ~15);
    const int tree_bytes = (Gmax.total * 4 + 15) & ~15;
    uint16_t* deg = reinterpret_cast<uint16_t*>(base);
    uint32_t* tree = reinterpret_cast<uint32_t*>(base + deg_bytes);
    int* misc = reinterpret_cast<int*>(base + deg_bytes + tree_bytes);
    const int slot_id = blockIdx.x * P.warps_per_cta + wib;
    uint8_t* slot = P.slots + (size_t)slot_id * P.slot.bytes;
    const uint64_t total = P.prefix[P.count];
    for (;;) {
        unsigned long long gq = 0;
        if (lane == 0) gq = atomicAdd(P.work, 1ull);
        gq = __shfl_sync(kFull, gq, 0);
        if (gq >= total) break;
        int lo = 0, hi = P.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.prefix[mid] <= gq) lo = mid; else hi = mid - 1;
        }
        run_trajectory<Real, TRACE>(P, lo, gq, gq - P.prefix[lo], deg, tree, misc, slot, lane);
    }
}

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
    double mx = -INFINITY, alive = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double v = log_x[i];
        if (v > -INFINITY) { mx = fmax(mx, v); alive += 1; }
    }
    mx = block_reduce_max(mx, sh);
    alive = block_reduce_sum(alive, sh);
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
    const double cnt = (double)(hi - lo);
    double m2 = 0;
    if (mx > -INFINITY) {
        const double mean = s1 / cnt;
        for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const double v = log_x[i];
            const double y = v > -INFINITY ? exp(v - mx) : 0.0;
            m2 += (y - mean) * (y - mean);
        }
    }
    m2 = block_reduce_sum(m2, sh);
    if (threadIdx.x == 0) {
        StatsPartial& p = parts[(size_t)k * chunks + ch];
        p.c = mx; p.s1 = s1; p.s2 = s2; p.m2 = m2;
        p.cnt = hi - lo;
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

cudaError_t launch_prepare(DevMatrix* d_mats, const DevInput* d_in, int count, Sched s, int, uint32_t* status,
                           cudaStream_t st)
{
    if (s.precision == 1) prepare_kernel<double><<<count, 1024, 0, st>>>(d_mats, d_in, s, status);
    else prepare_kernel<float><<<count, 1024, 0, st>>>(d_mats, d_in, s, status);
    return cudaGetLastError();
}

template <typename Real, bool TRACE>
static cudaError_t launch_traj_t(const TrajParams& p, int grid, cudaStream_t st)
{
    const int smem = p.smem_per_warp * p.warps_per_cta;
    cudaError_t e = cudaFuncSetAttribute(traj_kernel<Real, TRACE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    traj_kernel<Real, TRACE><<<grid, p.warps_per_cta * 32, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_trajectories(const TrajParams& p, int grid, bool trace, cudaStream_t st)
{
    if (p.s.precision == 1) return trace ? launch_traj_t<double, true>(p, grid, st) : launch_traj_t<double, false>(p, grid, st);
    return trace ? launch_traj_t<float, true>(p, grid, st) : launch_traj_t<float, false>(p, grid, st);
}

cudaError_t traj_occupancy(bool fp64, bool trace, int warps_per_cta, int smem, int* ctas_per_sm)
{
    const void* f = fp64 ? (trace ? (const void*)traj_kernel<double, true> : (const void*)traj_kernel<double, false>)
                         : (trace ? (const void*)traj_kernel<float, true> : (const void*)traj_kernel<float, false>);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, f, warps_per_cta * 32, smem);
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
