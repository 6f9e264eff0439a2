// pm_traj.cu -- the trajectory kernel (Algorithm 2, one trajectory per group
// of g warps).
//
// Per step the group's leader warp
//   - picks the active row or column of least (live degree, unified id)
//     from a 32-ary tree of packed keys (two-sided minimum degree, Sec. 3.2),
//   - scans the picked vertex's adjacency (one lane per entry), forms the
//     integer proposal weights of Eq. 3 and draws the partner with Philox,
//   - multiplies X by B_vu / q(u|v) (kept as mantissa/exponent pairs),
//   - eliminates the pair: decrements the live degrees of both neighbour
//     lists and lowers / repairs the tree entries above them,
//   - decides the DM policy (All / Thrs / Trck) and the number of full SK
//     iterations (Fixed / Adaptive), or runs the Local repair of Eq. 5;
// then the whole group runs the InnerDM degree rebuild and the full SK
// iterations (one thread per column, then per row; every sum is taken in
// adjacency order so the result is fixed by IEEE arithmetic alone).
//
// A persistent CTA takes chunks of trajectories of one matrix at a time and,
// when the plan says so, stages that matrix's adjacency (uint16 indices) in
// shared memory for all its groups.  Plans without inner SK or DM may run
// two trajectories per warp instead (pm_pair.cuh); a launch of such plans
// only, for the scaled or uniform proposal, uses the 24-warp pair-only
// kernel.  In the PM_DEBUG build the matrix is read through checked views.
#include <cmath>
#include "pm_device.cuh"
#include "pm_dm.cuh"
#include "pm_mlp.cuh"

namespace pm {

namespace {

enum { VR_ROW = 1 };
enum { SKP_NONE = 0, SKP_FIXED = 1, SKP_ADAPTIVE = 2, SKP_LOCAL = 3 };
enum { DMP_NONE = 0, DMP_ALL = 1, DMP_THRS = 2, DMP_TRCK = 3 };

template <typename Idx>
struct MV {
    int n;
    ChkPtr<int> rp;   // row pointers
    ChkPtr<int> cp;   // column pointers
    ChkPtr<Idx> ci;   // column index of each row entry
    ChkPtr<Idx> ri;   // row index of each column entry
    ChkPtr<int> ce;   // row-entry id of each column entry (DM masks)
    const float* rv;  // values in row order or nullptr
    const float* cv;  // values in column order or nullptr
};

// the view of B0 a trajectory reads (checked arrays in the PM_DEBUG build)
template <typename Idx>
__device__ __forceinline__ MV<Idx> make_mv(int n, int m, const int* rp, const int* cp, const Idx* ci, const Idx* ri,
                                           const int* ce, const float* rv, const float* cv)
{
#ifdef PM_DEBUG
    const uint32_t n1 = (uint32_t)n + 1u, m0 = (uint32_t)m, m1 = (uint32_t)m + 1u;
    return MV<Idx>{n, {rp, n1, m1}, {cp, n1, m1}, {ci, m0, (uint32_t)n}, {ri, m0, (uint32_t)n}, {ce, m0, m0}, rv, cv};
#else
    (void)m;
    return MV<Idx>{n, rp, cp, ci, ri, ce, rv, cv};
#endif
}

__device__ __forceinline__ size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

struct Grp {
    int g, nthr, tid, wig, lane, bar;
    int* misc;
    bool gdm;  // the group shares the DM's component step (state in global memory, g > 1)
};

__device__ __forceinline__ void gsync(const Grp& G)
{
    if (G.g == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(G.bar), "r"(G.nthr) : "memory");
}

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

// ---- minimum-degree tree ----
// (the level loops run over the compile-time maximum so the geometry arrays
// are indexed statically and stay in registers)
__device__ __forceinline__ void tree_lower(uint32_t* tree, const TreeGeom& T, int x, uint32_t d)
{
    const uint32_t key = ((d < T.dcap ? d : T.dcap) << T.idb) | (uint32_t)x;
#pragma unroll
    for (int l = 1; l <= kMaxTreeLevels; ++l)
        if (l <= T.nlev) atomicMin(&tree[T.off[l] + (x >> (5 * l))], key);
}

// recompute the tree entries above leaves x and y (two independent chains)
__device__ void tree_fix2(const uint16_t* deg, uint32_t* tree, const TreeGeom& T, int x, int y, int lane)
{
#pragma unroll
    for (int l = 1; l <= kMaxTreeLevels; ++l) {
        if (l > T.nlev) break;
        const int gx = x >> (5 * l), gy = y >> (5 * l);
        const bool two = gy != gx;
        const int cx = gx * 32 + lane, cy = gy * 32 + lane;
        uint32_t kx = 0xFFFFFFFFu, ky = 0xFFFFFFFFu;
        if (cx < T.size[l - 1]) kx = (l == 1) ? leaf_key(deg, cx, T) : tree[T.off[l - 1] + cx];
        if (two && cy < T.size[l - 1]) ky = (l == 1) ? leaf_key(deg, cy, T) : tree[T.off[l - 1] + cy];
        kx = __reduce_min_sync(kFull, kx);
        ky = __reduce_min_sync(kFull, ky);
        if (lane == 0) {
            tree[T.off[l] + gx] = kx;
            if (two) tree[T.off[l] + gy] = ky;
        }
        __syncwarp();
    }
}

__device__ void tree_build(const uint16_t* deg, uint32_t* tree, const TreeGeom& T, int lane)
{
    for (int l = 1; l <= T.nlev; ++l) {
        for (int gi = lane; gi < T.size[l]; gi += 32) {
            uint32_t best = 0xFFFFFFFFu;
            for (int q = 0; q < 32; ++q) {
                const int c = gi * 32 + q;
                if (c >= T.size[l - 1]) break;
                const uint32_t key = (l == 1) ? leaf_key(deg, c, T) : tree[T.off[l - 1] + c];
                best = key < best ? key : best;
            }
            tree[T.off[l] + gi] = best;
        }
        __syncwarp();
    }
}

// the same with the whole group (large n): level by level, one thread per
// upper entry, a group barrier between levels
template <class Sync>
__device__ void tree_build_group(const uint16_t* deg, uint32_t* tree, const TreeGeom& T, int tid, int nthr, Sync sync)
{
    for (int l = 1; l <= T.nlev; ++l) {
        for (int gi = tid; gi < T.size[l]; gi += nthr) {
            uint32_t best = 0xFFFFFFFFu;
            for (int q = 0; q < 32; ++q) {
                const int c = gi * 32 + q;
                if (c >= T.size[l - 1]) break;
                const uint32_t key = (l == 1) ? leaf_key(deg, c, T) : tree[T.off[l - 1] + c];
                best = key < best ? key : best;
            }
            tree[T.off[l] + gi] = best;
        }
        sync();
    }
}

__device__ __forceinline__ int md_pick(const uint16_t* deg, const uint32_t* tree, const TreeGeom& T, int lane)
{
    uint32_t key = 0xFFFFFFFFu;
    int top_off = 0, top_size = T.n2;
#pragma unroll
    for (int l = 1; l <= kMaxTreeLevels; ++l)
        if (l == T.nlev) { top_off = T.off[l]; top_size = T.size[l]; }
    if (T.nlev == 0) {
        if (lane < T.n2) key = leaf_key(deg, lane, T);
    } else if (lane < top_size) {
        key = tree[top_off + lane];
    }
    key = __reduce_min_sync(kFull, key);
    if ((key >> T.idb) < T.dcap) return (int)(key & ((1u << T.idb) - 1u));
    unsigned long long best = ~0ull;  // saturated degree field: exact scan
    for (int x = lane; x < T.n2; x += 32) {
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

template <typename Idx>
__device__ __forceinline__ bool entry_live(const uint16_t* deg, const uint8_t* mask, const MV<Idx>& V, bool row_list,
                                           int e, int pid)
{
    if (deg[pid] == kInact) return false;
    if (!mask) return true;
    return mask[row_list ? e : V.ce[e]] != 0;
}

// ---- SK sums in adjacency order.  Eliminated rows and columns carry a zero
// scale in the per-trajectory vectors, so an entry to an inactive vertex
// adds B * 0 = +0, which leaves the sum bit-identical to skipping it (every
// partial sum is >= +0); only DM-removed edges need a test.  Unrolled by four
// so the gathers of one vertex are in flight together. ----
template <typename Real, typename Idx>
__device__ __forceinline__ Real col_sum(const MV<Idx>& V, const uint8_t* mask, const Real* r, int j)
{
    const int b = V.cp[j], e = V.cp[j + 1];
    Real sum = 0;
    int k = b;
    for (; k + 4 <= e; k += 4) {
        Real t0 = r[V.ri[k]], t1 = r[V.ri[k + 1]], t2 = r[V.ri[k + 2]], t3 = r[V.ri[k + 3]];
        if (V.cv) {
            t0 = RA<Real>::mul((Real)__ldg(V.cv + k), t0);
            t1 = RA<Real>::mul((Real)__ldg(V.cv + k + 1), t1);
            t2 = RA<Real>::mul((Real)__ldg(V.cv + k + 2), t2);
            t3 = RA<Real>::mul((Real)__ldg(V.cv + k + 3), t3);
        }
        if (mask) {
            if (!mask[V.ce[k]]) t0 = 0;
            if (!mask[V.ce[k + 1]]) t1 = 0;
            if (!mask[V.ce[k + 2]]) t2 = 0;
            if (!mask[V.ce[k + 3]]) t3 = 0;
        }
        sum = RA<Real>::add(sum, t0);
        sum = RA<Real>::add(sum, t1);
        sum = RA<Real>::add(sum, t2);
        sum = RA<Real>::add(sum, t3);
    }
    for (; k < e; ++k) {
        Real t = r[V.ri[k]];
        if (V.cv) t = RA<Real>::mul((Real)__ldg(V.cv + k), t);
        if (mask && !mask[V.ce[k]]) t = 0;
        sum = RA<Real>::add(sum, t);
    }
    return sum;
}

template <typename Real, typename Idx>
__device__ __forceinline__ Real row_sum(const MV<Idx>& V, const uint8_t* mask, const Real* c, int i)
{
    const int b = V.rp[i], e = V.rp[i + 1];
    Real sum = 0;
    int k = b;
    for (; k + 4 <= e; k += 4) {
        Real t0 = c[V.ci[k]], t1 = c[V.ci[k + 1]], t2 = c[V.ci[k + 2]], t3 = c[V.ci[k + 3]];
        if (V.rv) {
            t0 = RA<Real>::mul((Real)__ldg(V.rv + k), t0);
            t1 = RA<Real>::mul((Real)__ldg(V.rv + k + 1), t1);
            t2 = RA<Real>::mul((Real)__ldg(V.rv + k + 2), t2);
            t3 = RA<Real>::mul((Real)__ldg(V.rv + k + 3), t3);
        }
        if (mask) {
            if (!mask[k]) t0 = 0;
            if (!mask[k + 1]) t1 = 0;
            if (!mask[k + 2]) t2 = 0;
            if (!mask[k + 3]) t3 = 0;
        }
        sum = RA<Real>::add(sum, t0);
        sum = RA<Real>::add(sum, t1);
        sum = RA<Real>::add(sum, t2);
        sum = RA<Real>::add(sum, t3);
    }
    for (; k < e; ++k) {
        Real t = c[V.ci[k]];
        if (V.rv) t = RA<Real>::mul((Real)__ldg(V.rv + k), t);
        if (mask && !mask[k]) t = 0;
        sum = RA<Real>::add(sum, t);
    }
    return sum;
}

// Compact the vertices this warp owns (a contiguous id range) that an SK
// iteration updates: active with at least one live edge.  Degrees do not
// change during the iterations of a step, so the lists serve all of them.
template <typename ListT>
__device__ __forceinline__ int compact_owned(const uint16_t* deg, int first, int last, int base_id, ListT* out,
                                             int lane)
{
    int cnt = 0;
    for (int x0 = first; x0 < last; x0 += 32) {
        const int x = x0 + lane;
        bool keep = false;
        if (x < last) {
            const uint16_t d = deg[base_id + x];
            keep = d != kInact && d != 0;
        }
        const unsigned km = __ballot_sync(kFull, keep);
        if (keep) out[cnt + __popc(km & ((1u << lane) - 1u))] = (ListT)x;
        cnt += __popc(km);
    }
    return cnt;
}

// one full SK iteration on the residual by the whole group (Sec. 3.3):
// columns from r, then rows from the new c, each warp over its own list
template <typename Real, typename Idx, typename ListT>
__device__ void sk_iteration(const MV<Idx>& V, const uint8_t* mask, Real* r, Real* c, const ListT* lc, int nc,
                             const ListT* lr, int nr, const Grp& G)
{
    for (int q = G.lane; q < nc; q += 32) {
        const int j = lc[q];
        c[j] = RA<Real>::rcp(col_sum<Real, Idx>(V, mask, r, j));
    }
    gsync(G);
    for (int q = G.lane; q < nr; q += 32) {
        const int i = lr[q];
        r[i] = RA<Real>::rcp(row_sum<Real, Idx>(V, mask, c, i));
    }
    gsync(G);
}

// Bounded-work Local repair (cap L > 0; Sec. 3.3 leaves the design open): the
// new scale of a vertex whose list in B^(0) (the matrix the trajectories run
// on, compacted after the initial DM) holds more than L entries, from the L
// list positions (o + q floor(len / L)) mod len, o = u mod len: the live
// sampled terms summed in sample order, times deg / (their count); no live
// sample keeps the old scale.  Explicit liveness tests (the count matters).
template <typename Real, typename Idx>
__device__ Real sampled_scale(const MV<Idx>& V, const uint16_t* deg, const uint8_t* mask, const Real* sc, bool row,
                              int x, uint64_t u, int L, Real old)
{
    const int n = V.n;
    const int b = row ? V.rp[x] : V.cp[x];
    const int len = (row ? V.rp[x + 1] : V.cp[x + 1]) - b;
    const int s = len / L;
    const int o = (int)(u % (uint64_t)len);
    Real acc = 0;
    int cnt = 0;
    for (int q = 0; q < L; ++q) {
        const int k = b + (int)(((long long)o + (long long)q * s) % len);
        int p, e;
        if (row) { p = n + (int)V.ci[k]; e = k; }
        else { p = (int)V.ri[k]; e = V.ce[k]; }
        if (deg[p] == kInact || (mask && !mask[e])) continue;
        Real t = sc[row ? p - n : p];
        const float* vals = row ? V.rv : V.cv;
        if (vals) t = RA<Real>::mul((Real)__ldg(vals + k), t);
        acc = RA<Real>::add(acc, t);
        ++cnt;
    }
    if (cnt == 0) return old;
    const Real est = RA<Real>::div(RA<Real>::mul(acc, (Real)deg[row ? x : n + x]), (Real)cnt);
    return RA<Real>::rcp(est);
}

// Local repair (Eq. 5) by the leader warp.  lr: N_t(C)\{R} (rows), lc:
// N_t(R)\{C} (columns).  R_loc = lr U N_{t+1}(lc), C_loc = lc U N_{t+1}(lr).
// New row scales read the old c and are staged (deduplicated by stamp);
// column scales read the old r and are written in place; staged rows commit
// last.  With a cap L > 0, lists longer than L are not expanded and their
// sums are sampled (sampled_scale, u the step's sampling word).  Returns the
// number of staged rows.
template <typename Real, typename Idx>
__device__ int local_repair(const MV<Idx>& V, const uint16_t* deg, const uint8_t* mask, Real* r, Real* c,
                            const int* lr, int nr, const int* lc, int nc, int* stamp, int st, int* tmp_id,
                            Real* tmp_val, int* tmp_cnt, int lane, int L, uint64_t u)
{
    const int n = V.n;
    if (lane == 0) *tmp_cnt = 0;
    __syncwarp();
    auto stage_row = [&](int i) {
        if (atomicExch(&stamp[i], st) == st) return;
        Real v;
        if (deg[i] == 0) v = r[i];
        else if (L > 0 && V.rp[i + 1] - V.rp[i] > L) v = sampled_scale<Real, Idx>(V, deg, mask, c, true, i, u, L, r[i]);
        else v = RA<Real>::rcp(row_sum<Real, Idx>(V, mask, c, i));
        const int q = atomicAdd(tmp_cnt, 1);
        tmp_id[q] = i;
        tmp_val[q] = v;
    };
    for (int q = lane; q < nr; q += 32) stage_row(lr[q]);
    for (int q = lane; q < nc; q += 32) {
        const int j = lc[q];
        if (L > 0 && V.cp[j + 1] - V.cp[j] > L) continue;
        for (int k = V.cp[j]; k < V.cp[j + 1]; ++k) {
            const int i = V.ri[k];
            if (deg[i] == kInact || (mask && !mask[V.ce[k]])) continue;
            stage_row(i);
        }
    }
    __syncwarp();
    auto col_new = [&](int j) {
        if (deg[n + j] == 0) return;
        if (L > 0 && V.cp[j + 1] - V.cp[j] > L) c[j] = sampled_scale<Real, Idx>(V, deg, mask, r, false, j, u, L, c[j]);
        else c[j] = RA<Real>::rcp(col_sum<Real, Idx>(V, mask, r, j));
    };
    for (int q = lane; q < nc; q += 32) col_new(lc[q]);
    for (int q = lane; q < nr; q += 32) {
        const int i = lr[q];
        if (L > 0 && V.rp[i + 1] - V.rp[i] > L) continue;
        for (int k = V.rp[i]; k < V.rp[i + 1]; ++k) {
            const int j = V.ci[k];
            if (deg[n + j] == kInact || (mask && !mask[k])) continue;
            col_new(j);
        }
    }
    __syncwarp();
    const int cnt = *tmp_cnt;
    for (int q = lane; q < cnt; q += 32) r[tmp_id[q]] = tmp_val[q];
    __syncwarp();
    return cnt;
}

template <typename Real, typename Idx>
__device__ __forceinline__ Real cand_score(const MV<Idx>& V, bool vrow, int e, int p, const Real* r, const Real* c)
{
    const float* vals = vrow ? V.rv : V.cv;
    const Real sc = vrow ? c[p] : r[p];
    Real s = vals ? RA<Real>::mul((Real)__ldg(vals + e), sc) : sc;
    if (!(s >= (Real)0)) s = 0;
    return s;
}

// Per-edge features of candidate p of the picked vertex v at step t (the
// learned proposal's inputs): log1p deg(v), log1p deg(p),
// log1p of the degree sum over v's live candidates, log1p of the degree sum
// over p's live neighbours, t / n, ln of the outer scales of v and p, ln B_vp.
// Sum, over the live neighbours of each live lane's candidate p, of their live
// degrees: the whole warp scans one candidate's adjacency at a time (one lane
// per entry, an integer reduction), so the cost is one pass per candidate
// instead of a serial loop per lane.  Integer sums: the result does not depend
// on the order.
template <typename Idx>
__device__ __forceinline__ int neighbour_degree_sum(const MV<Idx>& V, const uint16_t* deg, const uint8_t* mask,
                                                    bool vrow, int pp, bool live, int lane)
{
    const int n = V.n;
    int mine = 0;
    unsigned lm = __ballot_sync(kFull, live);
    while (lm) {
        const int src = __ffs(lm) - 1;
        lm &= lm - 1u;
        const int p = __shfl_sync(kFull, pp, src);
        const int b = vrow ? V.cp[p] : V.rp[p];
        const int en = vrow ? V.cp[p + 1] : V.rp[p + 1];
        unsigned acc = 0;
        for (int k = b + lane; k < en; k += 32) {
            if (vrow) {  // p is a column: its live rows
                const int i = V.ri[k];
                const unsigned d = deg[i];
                if (d != kInact && (!mask || mask[V.ce[k]])) acc += d;
            } else {     // p is a row: its live columns
                const int j = V.ci[k];
                const unsigned d = deg[n + j];
                if (d != kInact && (!mask || mask[k])) acc += d;
            }
        }
        const unsigned tot = __reduce_add_sync(kFull, acc);
        if (lane == src) mine = (int)tot;
    }
    return mine;
}

// the global inputs of a candidate's features (outer scale of p, entry B_vp),
// loaded as soon as p is known so the loads overlap the neighbour scan
struct CandLoads {
    float sl, bv;
};
template <typename Idx>
__device__ __forceinline__ CandLoads cand_loads(const MV<Idx>& V, const DevMatrix* Mp, bool vrow, int e, int p,
                                                bool live)
{
    CandLoads c{1.0f, 1.0f};
    if (!live) return c;
    const float* s0 = reinterpret_cast<const float*>(vrow ? Mp->c0 : Mp->r0);
    c.sl = __ldg(s0 + p);
    const float* vals = vrow ? V.rv : V.cv;
    if (vals) c.bv = __ldg(vals + e);
    return c;
}

// The same sums in one warp pass over all candidates' adjacency entries at
// once (lane f takes flat entry f of the concatenated lists); the per-
// candidate sums are formed by shared-memory atomics in `acc` (32 ints).
// Integer sums: identical to neighbour_degree_sum.
template <typename Idx>
__device__ __forceinline__ int neighbour_degree_sum_flat(const MV<Idx>& V, const uint16_t* deg, const uint8_t* mask,
                                                         bool vrow, int pp, bool live, int lane, int* acc,
                                                         int& entries)
{
    const int n = V.n;
    int b = 0, len = 0;
    if (live) {
        b = vrow ? V.cp[pp] : V.rp[pp];
        len = (vrow ? V.cp[pp + 1] : V.rp[pp + 1]) - b;
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - len;
    const int total = __shfl_sync(kFull, incl, 31);
    entries = total;
    acc[lane] = 0;
    __syncwarp();
    const bool has = live && len > 0;
    const unsigned lm = __ballot_sync(kFull, has);
    for (int base = 0; base < total; base += 32) {
        const int f = base + lane;
        // the candidate whose range holds f is the last one starting at or
        // before f: candidates starting before this chunk, plus the starts
        // inside it up to f (ranges are contiguous in lane order)
        const unsigned before = __ballot_sync(kFull, has && excl < base);
        const unsigned starts =
            __reduce_or_sync(kFull, (has && excl >= base && excl < base + 32) ? 1u << (excl - base) : 0u);
        const int rank = __popc(before) + __popc(starts & (0xFFFFFFFFu >> (31 - lane)));
        int owner = -1, pos = 0;
        if (f < total) owner = (int)__fns(lm, 0, rank);  // lane of the rank-th candidate
        const int src = owner >= 0 ? owner : 0;
        const int oe = __shfl_sync(kFull, excl, src), ob = __shfl_sync(kFull, b, src);
        if (owner >= 0) pos = ob + (f - oe);
        if (owner >= 0) {
            unsigned d;
            bool ok;
            if (vrow) {  // the candidate is a column: its live rows
                const int i = V.ri[pos];
                d = deg[i];
                ok = d != kInact && (!mask || mask[V.ce[pos]]);
            } else {     // the candidate is a row: its live columns
                const int j = V.ci[pos];
                d = deg[n + j];
                ok = d != kInact && (!mask || mask[pos]);
            }
            if (ok) atomicAdd(acc + owner, (int)d);
        }
    }
    __syncwarp();
    const int mine = acc[lane];
    __syncwarp();
    return mine;
}

template <typename Idx>
__device__ __forceinline__ void cand_features(const MV<Idx>& V, const uint16_t* deg, int t, bool vrow, int p,
                                              float sum_v, int sum_l, float dv, float lsv, const CandLoads& cl,
                                              float (&f)[8])
{
    const int n = V.n;
    const float sl = cl.sl, bv = cl.bv;
    const float* vals = vrow ? V.rv : V.cv;
    // fast logarithms (about 1e-6 relative): 1 + an integer count is exact in binary32
    f[0] = __logf(1.0f + dv);
    f[1] = __logf(1.0f + (float)deg[p + (vrow ? n : 0)]);
    f[2] = __logf(1.0f + sum_v);
    f[3] = __logf(1.0f + (float)sum_l);
    f[4] = __fdiv_rn((float)t, (float)n);
    f[5] = lsv;
    f[6] = __logf(sl);
    f[7] = vals ? __logf(bv) : 0.0f;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// misc slots of a group (two step buffers so a fast leader never overwrites
// values a slower warp of its group is still reading)
enum { M_DEAD = 0, M_NIT = 1, M_DM = 2, M_CNTR = 3, M_CNTC = 4, M_STRIDE = 8, M_TMP = 16, M_TRAJ = 17, M_DMOK = 18,
       M_DMSH = 20 /* 8 ints: the group DM's counters */ };

// MODE: 0 scaled proposal, 1 learned proposal, 2 recording of (features, SK target) pairs
template <typename Real, typename Idx, bool TRACE, int MODE, typename ListT>
__device__ void run_group(const TrajParams& P, const DevMatrix* Mp, const MV<Idx>& V, int k, uint64_t gq,
                          uint64_t local, uint16_t* deg, uint32_t* tree, Real* r_sm, ListT* lists, uint16_t* feat,
                          const DevModel* Ms, uint8_t* slot, int* dm_sm, uint8_t* mask_sm, const Grp& G)
{
    constexpr bool model = MODE == 1;
    constexpr bool rec = MODE == 2;
    const int n = V.n;
    const int lane = G.lane;
    const bool leader = G.wig == 0;
    const uint64_t traj = P.first_traj + local;
    const uint32_t midx = (uint32_t)Mp->idx;
    const Sched& S = P.s;
    const TreeGeom T = tree_geom(n);
    if (TRACE && leader) {
        for (int q = lane; q < 2 * n; q += 32) P.chosen[gq * 2 * n + q] = -1;
        for (int q = lane; q < n; q += 32) P.deg_v[gq * n + q] = -1;
    }
    if (!Mp->ok) {
        if (leader && lane == 0) {
            P.log_x[gq] = -INFINITY;
            if (TRACE) P.dead_step[gq] = 0;
        }
        gsync(G);
        return;
    }
    const bool inner_sk = S.sk != SKP_NONE;
    const bool use_dm = S.dm != DMP_NONE;
    const bool use_local = S.sk == SKP_LOCAL;

    // trajectory state from the shared initial state
    {
        const uint4* src = reinterpret_cast<const uint4*>(Mp->deg0);
        uint4* dst = reinterpret_cast<uint4*>(deg);
        const int nv = (2 * n + 7) / 8;
        for (int q = G.tid; q < nv; q += G.nthr) dst[q] = __ldg(src + q);
        for (int q = G.tid; q < T.total; q += G.nthr) tree[q] = __ldg(Mp->tree0 + q);
    }
    Real* r;
    Real* c;
    if (inner_sk) {
        if (r_sm) {
            r = r_sm;
            c = reinterpret_cast<Real*>(reinterpret_cast<uint8_t*>(r_sm) + a16((size_t)n * sizeof(Real)));
        } else {
            r = reinterpret_cast<Real*>(slot + P.slot.r);
            c = reinterpret_cast<Real*>(slot + P.slot.c);
        }
        const Real* r0 = reinterpret_cast<const Real*>(Mp->r0);
        const Real* c0 = reinterpret_cast<const Real*>(Mp->c0);
        for (int q = G.tid; q < n; q += G.nthr) { r[q] = __ldg(r0 + q); c[q] = __ldg(c0 + q); }
    } else {
        r = reinterpret_cast<Real*>(Mp->r0);
        c = reinterpret_cast<Real*>(Mp->c0);
    }
    uint8_t* mask = nullptr;
    int* dmws = nullptr;
    bool dm_matched = false;  // the DM workspace holds this trajectory's last perfect matching
    if (use_dm) {
        mask = mask_sm ? mask_sm : slot + P.slot.mask;
        dmws = dm_sm ? dm_sm : reinterpret_cast<int*>(slot + P.slot.dm);
        const int m = Mp->m;
        for (int q = G.tid; q < m; q += G.nthr) mask[q] = 1;
        if (Mp->matched) {  // start from the initial DM's perfect matching of B0
            for (int q = G.tid; q < 2 * n; q += G.nthr) dmws[q] = __ldg(Mp->dm_ws + q);
            dm_matched = true;
        }
    }
    int *stamp = nullptr, *tmp_id = nullptr, *list_r = nullptr, *list_c = nullptr;
    Real* tmp_val = nullptr;
    if (use_local) {
        stamp = reinterpret_cast<int*>(slot + P.slot.stamp);
        tmp_id = reinterpret_cast<int*>(slot + P.slot.tmp_id);
        tmp_val = reinterpret_cast<Real*>(slot + P.slot.tmp_val);
        list_r = reinterpret_cast<int*>(slot + P.slot.list_r);
        list_c = reinterpret_cast<int*>(slot + P.slot.list_c);
        for (int q = G.tid; q < n; q += G.nthr) stamp[q] = 0;
    }
    gsync(G);

    const bool uniform = Mp->unit_scale && !inner_sk;
    const Real theta = (Real)S.theta;
    // leader-lane state: X = num / den
    Mant64 num, den;
    Real track = 1;
    unsigned n_dm = 0, n_full = 0, n_loc = 0;
    int dead_step = -1;
    // algorithmic bytes of the trajectory: 16 B per vertex for the initial
    // degrees and minimum-degree structure; then per step the counts below
    uint64_t alg_bytes = (uint64_t)16 * n;
    const uint64_t t_begin = (leader && lane == 0) ? global_ns() : 0;
    uint64_t mlp_rows = 0;  // network evaluations of live candidates (learned proposal)
    int m_live = Mp->m;

    bool abandoned = false;
    for (int t = 0; t < n; ++t) {
        int* mb = G.misc + (t & 1) * M_STRIDE;
        if (leader) {
            int dead = 0, nit = 0, run_dm = 0, cnt_r = 0, cnt_c = 0;
            if (P.hard_ns && (t & 63) == 0) {  // far past the budget: leave this trajectory out
                int over = 0;
                if (lane == 0) {
                    const unsigned long long t0 = *reinterpret_cast<volatile unsigned long long*>(P.t_start);
                    over = t0 && global_ns() - t0 > P.hard_ns;
                }
                if (__shfl_sync(kFull, over, 0)) {
                    if (lane == 0) atomicOr(P.status, ST_TIMEOUT);
                    abandoned = true;
                    dead = 1;
                }
            }
            if (!dead) do {  // the sequential part of step t (breaks out on death)
                // draw 0 of this step depends on (seed, trajectory, step) only:
                // computed first, it overlaps the pick and the candidate scan
                const uint64_t u0 = draw_u64(P.seed, traj, midx, (uint32_t)t, 0);
                int v = (S.vertex_rule == VR_ROW) ? t : md_pick(deg, tree, T, lane);
                PM_CLAMP(v, 2 * n);
                const int dv = deg[v];
                if (TRACE && lane == 0) P.deg_v[gq * n + t] = dv;
                if (dv == 0) { dead = 1; break; }
                const bool vrow = v < n;
                const int vi = vrow ? v : v - n;
                const int beg = (vrow ? V.rp : V.cp)[vi];
                const int end = (vrow ? V.rp : V.cp)[vi + 1];
                const auto adj = vrow ? V.ci : V.ri;
                const int poff = vrow ? n : 0;
                const int kq = 40 - bitlen((uint32_t)dv);
                const int len = end - beg;

                uint64_t W = 0, w_sel = 0;
                int sel_e = -1, sel_p = -1;
                bool keep_live = false;
                int keep_pid = 0;
                uint64_t rr;
                // learned proposal: logits of the live candidates from their features
                float sum_v = 0.f;  // degree sum over v's live candidates (feature)
                float lsv = 0.f;    // ln of v's outer scale (feature)
                if (model || rec) {
                    const float* s0 = reinterpret_cast<const float*>(vrow ? Mp->r0 : Mp->c0);
                    const float sv0 = __ldg(s0 + vi);
                    int sv_i = 0;
                    for (int base = beg; base < end; base += 32) {
                        const int e = base + lane;
                        if (e < end) {
                            const int pid = (int)adj[e] + poff;
                            if (entry_live(deg, mask, V, vrow, e, pid)) sv_i += deg[pid];
                        }
                    }
#pragma unroll
                    for (int o = 16; o; o >>= 1) sv_i += __shfl_xor_sync(kFull, sv_i, o);
                    sum_v = (float)sv_i;
                    lsv = __logf(sv0);
                }
                // logits of the live candidates of one chunk: their features
                // go to rows 0..nl-1 of the tile (live order), the network
                // runs on 8 candidates at a time
                auto cand_logit = [&](int e, int pp, bool live) -> float {
                    const unsigned lmk = __ballot_sync(kFull, live);
                    const int nl = __popc(lmk);
                    const int li = __popc(lmk & ((1u << lane) - 1u));
                    const CandLoads cl = cand_loads<Idx>(V, Mp, vrow, e, pp, live);
                    // the feature tile doubles as the sums' scratch until the features are written
                    int entries = 0;
                    const int sum_l = neighbour_degree_sum_flat<Idx>(V, deg, mask, vrow, pp, live, lane,
                                                                     reinterpret_cast<int*>(feat), entries);
                    // features: each live candidate's list (index + degree, 8 B
                    // an entry) and pointers, its outer scale and entry value
                    alg_bytes += (uint64_t)8 * entries + (uint64_t)16 * nl;
                    if (live) {
                        float f[8];
                        cand_features<Idx>(V, deg, t, vrow, pp, sum_v, sum_l, (float)dv, lsv, cl, f);
                        uint4 lo;
                        lo.x = pack_bf16(f[0], f[1]);
                        lo.y = pack_bf16(f[2], f[3]);
                        lo.z = pack_bf16(f[4], f[5]);
                        lo.w = pack_bf16(f[6], f[7]);
                        *reinterpret_cast<uint4*>(feat + li * kFS) = lo;
                    }
                    __syncwarp();
                    float lg = 0.f;
                    for (int tile = 0; 8 * tile < nl; ++tile) {
                        const float y = mlp_infer8(Ms, feat + 8 * tile * kFS, lane);
                        const float yv = __shfl_sync(kFull, y, 4 * (li & 7));
                        if (live && (li >> 3) == tile) lg = yv;
                    }
                    __syncwarp();
                    return lg;
                };
                // score of a live candidate: B * c (scaled) or B * e^logit (learned)
                auto score = [&](int e, int pp, float lg) -> Real {
                    if (!model) return cand_score<Real, Idx>(V, vrow, e, pp, r, c);
                    const float* vals = vrow ? V.rv : V.cv;
                    const float ex = exp_score(lg);
                    Real sv = vals ? (Real)__fmul_rn(__ldg(vals + e), ex) : (Real)ex;
                    if (!(sv >= (Real)0)) sv = 0;
                    return sv;
                };
                // trace logits of the live candidates (learned proposal)
                auto side_outputs = [&](int e, int pp, bool live, float lg, int live_base) {
                    const unsigned lmk = __ballot_sync(kFull, live);
                    const int li = live_base + __popc(lmk & ((1u << lane) - 1u));
                    if (TRACE && model && live && li < P.logit_stride)
                        P.trace_logits[((size_t)gq * n + t) * P.logit_stride + li] = lg;
                    return __popc(lmk);
                };
                // recording of (features, SK target) pairs: a pair is kept
                // only if every value is finite (an SK scale can run to 0 or
                // infinity without total support); a step's kept pairs are
                // written together as one group, and only if there are at
                // least two (pass 1 counts them, pass 2 writes them)
                if (rec) {
                    auto pair_at = [&](int e, int pp, bool live, float (&f)[8], float& tgt) -> bool {
                        const CandLoads cl = cand_loads<Idx>(V, Mp, vrow, e, pp, live);
                        const int sum_l = neighbour_degree_sum<Idx>(V, deg, mask, vrow, pp, live, lane);
                        if (!live) return false;
                        cand_features<Idx>(V, deg, t, vrow, pp, sum_v, sum_l, (float)dv, lsv, cl, f);
                        const double sv_cur = vrow ? (double)r[vi] : (double)c[vi];
                        const double sl_cur = vrow ? (double)c[pp] : (double)r[pp];
                        tgt = (float)log(sv_cur * sl_cur);
                        bool keep = isfinite(tgt);
#pragma unroll
                        for (int q = 0; q < 8; ++q) keep = keep && isfinite(f[q]);
                        return keep;
                    };
                    int kept = 0;
                    for (int base = beg; base < end; base += 32) {
                        const int e = base + lane;
                        int pp = 0;
                        bool live = false;
                        if (e < end) {
                            pp = adj[e];
                            live = entry_live(deg, mask, V, vrow, e, pp + poff);
                        }
                        float f[8], tgt = 0.f;
                        kept += __popc(__ballot_sync(kFull, pair_at(e, pp, live, f, tgt)));
                    }
                    if (kept >= 2) {
                        unsigned long long b0 = 0;
                        if (lane == 0) b0 = atomicAdd(P.rec_count, (unsigned long long)kept);
                        b0 = __shfl_sync(kFull, b0, 0);
                        if (b0 + (unsigned long long)kept <= P.rec_cap) {
                            int qi = 0, li0 = 0;
                            for (int base = beg; base < end; base += 32) {
                                const int e = base + lane;
                                int pp = 0;
                                bool live = false;
                                if (e < end) {
                                    pp = adj[e];
                                    live = entry_live(deg, mask, V, vrow, e, pp + poff);
                                }
                                float f[8], tgt = 0.f;
                                const bool keep = pair_at(e, pp, live, f, tgt);
                                const unsigned lt = (1u << lane) - 1u;
                                const unsigned lmk = __ballot_sync(kFull, live), kmk = __ballot_sync(kFull, keep);
                                if (keep) {
                                    const int qq = qi + __popc(kmk & lt);
                                    const unsigned long long pos = b0 + (unsigned long long)qq;
                                    const int li = li0 + __popc(lmk & lt);
#pragma unroll
                                    for (int q = 0; q < 8; ++q) P.rec_feat[pos * 8 + q] = f[q];
                                    P.rec_target[pos] = tgt;
                                    P.rec_key[pos] = (traj << 28) | ((unsigned long long)t << 14) | (unsigned long long)li;
                                    P.rec_group[pos] = ((uint32_t)qq << 16) | (uint32_t)kept;
                                }
                                qi += __popc(kmk);
                                li0 += __popc(lmk);
                            }
                            if (lane == 0) atomicMax(P.rec_count + 1, b0 + (unsigned long long)kept);
                        }
                    }
                }
                // the network runs once per candidate: one pass over the list;
                // the logit of a single-chunk list stays in a register, longer
                // lists keep theirs in the group's slot
                float lg_reg = 0.f;
                float* lgbuf = model ? reinterpret_cast<float*>(slot + P.slot.logit) : nullptr;
                // a single live candidate is taken with probability 1 whatever
                // its score (W = w): no network evaluation, logit 0
                if (model && dv >= 2) {
                    int live_base = 0;
                    for (int base = beg; base < end; base += 32) {
                        const int e = base + lane;
                        int pp = 0;
                        bool live = false;
                        if (e < end) {
                            pp = adj[e];
                            live = entry_live(deg, mask, V, vrow, e, pp + poff);
                        }
                        const float lg = cand_logit(e, pp, live);
                        mlp_rows += __popc(__ballot_sync(kFull, live));
                        if (len > 32 && e < end) lgbuf[e - beg] = lg;
                        lg_reg = lg;
                        if (TRACE) live_base += side_outputs(e, pp, live, lg, live_base);
                    }
                }
                if (len <= 32) {
                    const int e = beg + lane;
                    const bool in = lane < len;
                    const int pp = in ? (int)adj[e] : 0;
                    const bool live = in && entry_live(deg, mask, V, vrow, e, pp + poff);
                    const unsigned lm = __ballot_sync(kFull, live);
                    const float lg = lg_reg;
                    uint64_t w, pre = 0;
                    if (uniform) {
                        w = live ? (1ull << kq) : 0ull;
                        W = (uint64_t)dv << kq;
                    } else {
                        const Real sv = live ? score(e, pp, lg) : (Real)0;
                        const Real smax = warp_max_nonneg(sv);
                        w = live ? quant_weight<Real>(sv, smax, kq) : 0ull;
                        pre = warp_incl_scan_u64(w, lane);  // W is its last element
                        W = __shfl_sync(kFull, pre, 31);
                    }
                    rr = uniform_below(W, u0, P.seed, traj, midx, (uint32_t)t);
                    if (rr == ~0ull) {
                        if (lane == 0) atomicOr(P.status, ST_RNG_EXHAUSTED);
                        dead = 1;
                        break;
                    }
                    int sl;
                    if (uniform) {
                        unsigned mm = lm;  // drop the first (rr >> kq) live lanes
                        for (int q = (int)(rr >> kq); q > 0; --q) mm &= mm - 1u;
                        sl = __ffs(mm) - 1;
                    } else {
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
                            int pp = 0;
                            bool live = false;
                            if (e < end) {
                                pp = adj[e];
                                live = entry_live(deg, mask, V, vrow, e, pp + poff);
                            }
                            const float lg = (model && dv >= 2 && e < end) ? lgbuf[e - beg] : 0.f;
                            if (live) sv = score(e, pp, lg);
                            const Real cm = warp_max_nonneg(sv);
                            smax = cm > smax ? cm : smax;
                        }
                        for (int base = beg; base < end; base += 32) {
                            const int e = base + lane;
                            uint64_t w = 0;
                            int pp = 0;
                            bool live = false;
                            if (e < end) {
                                pp = adj[e];
                                live = entry_live(deg, mask, V, vrow, e, pp + poff);
                            }
                            const float lg = (model && dv >= 2 && e < end) ? lgbuf[e - beg] : 0.f;
                            if (live) w = quant_weight<Real>(score(e, pp, lg), smax, kq);
                            W += warp_sum_u64(w);
                        }
                    } else {
                        W = (uint64_t)dv << kq;
                    }
                    rr = uniform_below(W, u0, P.seed, traj, midx, (uint32_t)t);
                    if (rr == ~0ull) {
                        if (lane == 0) atomicOr(P.status, ST_RNG_EXHAUSTED);
                        dead = 1;
                        break;
                    }
                    uint64_t carry = 0;
                    for (int base = beg; base < end; base += 32) {
                        const int e = base + lane;
                        int pp = 0;
                        bool live = false;
                        uint64_t w = 0;
                        if (e < end) {
                            pp = adj[e];
                            live = entry_live(deg, mask, V, vrow, e, pp + poff);
                        }
                        const float lg = (model && dv >= 2 && e < end) ? lgbuf[e - beg] : 0.f;
                        if (live) w = uniform ? (1ull << kq) : quant_weight<Real>(score(e, pp, lg), smax, kq);
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
                if (sel_p < 0 || sel_e < beg || sel_e >= end) {  // only with corrupt degrees
                    if (lane == 0) atomicOr(P.status, ST_INTERNAL);
                    dead = 1;
                    break;
                }
                const int R = vrow ? vi : sel_p;  // matched row
                const int C = vrow ? sel_p : vi;  // matched column
                if (TRACE && lane == 0) {
                    P.chosen[(gq * n + t) * 2 + 0] = v;
                    P.chosen[(gq * n + t) * 2 + 1] = sel_p + poff;
                }
                if (lane == 0) {  // X <- X * B_vu * W / w_u
                    num.mul(W);
                    const float* vals = vrow ? V.rv : V.cv;
                    if (vals) num.mul(__ldg(vals + sel_e));
                    den.mul(w_sel);
                }
                // z = r_R c_C drives the Thrs / Trck DM policies and Adaptive SK only
                const bool need_z = S.dm == DMP_THRS || S.dm == DMP_TRCK || S.sk == SKP_ADAPTIVE;
                const Real z = need_z ? RA<Real>::mul(r[R], c[C]) : (Real)1;

                // eliminate R and C (their per-trajectory scales become 0)
                __syncwarp();
                if (lane == 0) {
                    deg[R] = kInact;
                    deg[n + C] = kInact;
                    if (inner_sk) { r[R] = 0; c[C] = 0; }
                }
                __syncwarp();
                int* list_v = vrow ? list_c : list_r;
                int* list_u = vrow ? list_r : list_c;
                int cnt_v = 0, cnt_u = 0;
                if (len <= 32) {
                    if (keep_live) {
                        const uint32_t d = deg[keep_pid] - 1u;
                        deg[keep_pid] = (uint16_t)d;
                        tree_lower(tree, T, keep_pid, d);
                    }
                    const unsigned km = __ballot_sync(kFull, keep_live);
                    if (use_local && keep_live) list_v[__popc(km & ((1u << lane) - 1u))] = keep_pid - poff;
                    cnt_v = __popc(km);
                } else {
                    for (int base = beg; base < end; base += 32) {
                        const int e = base + lane;
                        bool live = false;
                        int pid = 0;
                        if (e < end) {
                            pid = (int)adj[e] + poff;
                            live = entry_live(deg, mask, V, vrow, e, pid);
                        }
                        if (live) {
                            const uint32_t d = deg[pid] - 1u;
                            deg[pid] = (uint16_t)d;
                            tree_lower(tree, T, pid, d);
                        }
                        const unsigned km = __ballot_sync(kFull, live);
                        if (use_local && live) list_v[cnt_v + __popc(km & ((1u << lane) - 1u))] = pid - poff;
                        cnt_v += __popc(km);
                    }
                }
                int ulen = 0;
                {  // the partner's list
                    const bool urow = !vrow;
                    const int ub = (urow ? V.rp : V.cp)[sel_p];
                    const int ue = (urow ? V.rp : V.cp)[sel_p + 1];
                    const auto uadj = urow ? V.ci : V.ri;
                    const int uoff = urow ? n : 0;
                    ulen = ue - ub;
                    for (int base = ub; base < ue; base += 32) {
                        const int e = base + lane;
                        bool live = false;
                        int pid = 0;
                        if (e < ue) {
                            pid = (int)uadj[e] + uoff;
                            live = entry_live(deg, mask, V, urow, e, pid);
                        }
                        if (live) {
                            const uint32_t d = deg[pid] - 1u;
                            deg[pid] = (uint16_t)d;
                            tree_lower(tree, T, pid, d);
                        }
                        const unsigned km = __ballot_sync(kFull, live);
                        if (use_local && live) list_u[cnt_u + __popc(km & ((1u << lane) - 1u))] = pid - uoff;
                        cnt_u += __popc(km);
                    }
                }
                cnt_r = vrow ? cnt_u : cnt_v;
                cnt_c = vrow ? cnt_v : cnt_u;
                m_live -= dv + cnt_u;
                // both eliminated lists: index + liveness check (8 B an entry)
                // and the two pointers of each list; 32 B per decrement
                // (degree read-modify-write + minimum-degree update); the
                // proposal's scale (and value) per candidate of v
                alg_bytes += (uint64_t)8 * (uint64_t)(len + ulen) + 16 + (uint64_t)32 * (uint64_t)(cnt_v + cnt_u);
                if (!uniform && !model) alg_bytes += (uint64_t)sizeof(Real) * (uint64_t)len;
                if ((vrow ? V.rv : V.cv) != nullptr) alg_bytes += (uint64_t)4 * (uint64_t)len;
                __syncwarp();
                if (S.vertex_rule != VR_ROW) tree_fix2(deg, tree, T, R, n + C, lane);
                track = RA<Real>::mul(track, z);
                if (t + 1 < n) {
                    run_dm = (S.dm == DMP_ALL) || (S.dm == DMP_THRS && z < theta) ||
                             (S.dm == DMP_TRCK && track < theta);
                    if (S.sk == SKP_FIXED) {
                        nit = S.K;
                    } else if (S.sk == SKP_ADAPTIVE) {
                        const Real b = RA<Real>::mul(RA<Real>::sub((Real)1, z), (Real)S.K);
                        nit = (b > (Real)0) ? (int)RA<Real>::ceil_(b) : 0;
                    }
                }
            } while (0);
            if (dead) dead_step = t;
            if (lane == 0) {
                mb[M_DEAD] = dead;
                mb[M_NIT] = nit;
                mb[M_DM] = run_dm;
                mb[M_CNTR] = cnt_r;
                mb[M_CNTC] = cnt_c;
            }
        }
        gsync(G);
        if (mb[M_DEAD]) break;
        if (t + 1 >= n) continue;
        if (mb[M_DM]) {
            if (leader) {
                ++n_dm;
                // a DM call: the matching repair and the SCC pass read each
                // live edge about once in each direction, plus per-vertex state
                alg_bytes += (uint64_t)16 * (uint64_t)m_live + (uint64_t)24 * (uint64_t)(2 * (n - t - 1));
            }
            const LiveTraj live{deg, mask, n};
            if (!G.gdm) {
                if (leader) {
                    const bool okdm = dm_warp(n, raw(V.rp), raw(V.ci), raw(V.cp), raw(V.ri), raw(V.ce), live, mask,
                                              dmws, lane, dm_matched);
                    dm_matched = okdm;
                    if (lane == 0) G.misc[M_DMOK] = okdm ? 1 : 0;
                }
            } else {
                // a group of warps (large n): the matching repair by group-
                // parallel augmenting searches (or, with no matching kept, the
                // leader warp's full matching), the component step's trimming
                // and giant-component searches on the whole group, Tarjan on
                // the leader for what is left, the mask on the whole group
                auto gs = [&] { gsync(G); };
                bool okdm;
                if (dm_matched) {
                    okdm = dm_repair_group(n, raw(V.rp), raw(V.ci), live, dmws, G.tid, G.nthr, G.misc + M_DMSH, gs);
                } else {
                    if (leader) {
                        const bool r = dm_match_warp(n, raw(V.rp), raw(V.ci), live, dmws, lane, false);
                        if (lane == 0) G.misc[M_DMOK] = r ? 1 : 0;
                    }
                    gsync(G);
                    okdm = G.misc[M_DMOK] != 0;
                    gsync(G);
                }
                dm_matched = okdm;
                if (leader && lane == 0) G.misc[M_DMOK] = okdm ? 1 : 0;
                if (okdm) {
                    const int nroots = dm_scc_group_prepass(n, raw(V.rp), raw(V.ci), raw(V.cp), raw(V.ri), raw(V.ce),
                                                            live, dmws, G.tid,
                                                            G.nthr, G.misc + M_DMSH, gs);
                    if (leader && nroots > 0) dm_tarjan_warp(n, raw(V.cp), raw(V.ri), raw(V.ce), live, dmws, lane, true, nroots);
                    gsync(G);
                    dm_mask_rows(n, raw(V.rp), raw(V.ci), live, mask, dmws, G.tid, G.nthr);
                }
            }
            gsync(G);
            if (!G.misc[M_DMOK]) {
                if (leader) dead_step = t;
                break;
            }
            // live degrees of the filtered child
            for (int x = G.tid; x < 2 * n; x += G.nthr) {
                if (deg[x] == kInact) continue;
                int d = 0;
                if (x < n) {
                    for (int e = V.rp[x]; e < V.rp[x + 1]; ++e) d += (mask[e] && deg[n + V.ci[e]] != kInact);
                } else {
                    const int j = x - n;
                    for (int kk = V.cp[j]; kk < V.cp[j + 1]; ++kk) d += (mask[V.ce[kk]] && deg[V.ri[kk]] != kInact);
                }
                deg[x] = (uint16_t)d;
            }
            gsync(G);
            if (G.gdm) {  // the whole group rebuilds the tree and counts the live edges
                tree_build_group(deg, tree, T, G.tid, G.nthr, [&] { gsync(G); });
                if (G.tid == 0) G.misc[M_DMSH] = 0;
                gsync(G);
                int ml = 0;
                for (int x = G.tid; x < n; x += G.nthr) ml += (deg[x] != kInact) ? deg[x] : 0;
                atomicAdd(G.misc + M_DMSH, ml);
                gsync(G);
                if (leader) {
                    track = 1;
                    m_live = G.misc[M_DMSH];
                }
            } else if (leader) {
                tree_build(deg, tree, T, lane);
                track = 1;
                int ml = 0;  // live edges of the child = sum of row degrees
                for (int x = lane; x < n; x += 32) ml += (deg[x] != kInact) ? deg[x] : 0;
#pragma unroll
                for (int o = 16; o; o >>= 1) ml += __shfl_xor_sync(kFull, ml, o);
                m_live = ml;
            }
            gsync(G);
        }
        const int nit = mb[M_NIT];
        if (nit > 0) {
            // this warp's share of the vertex ids, compacted to the ones updated
            const int per = (n + G.g - 1) / G.g;
            const int lo = min(n, G.wig * per), hi = min(n, lo + per);
            const int nc = compact_owned(deg, lo, hi, n, lists + lo, lane);
            const int nr = compact_owned(deg, lo, hi, 0, lists + n + lo, lane);
            __syncwarp();
            for (int q = 0; q < nit; ++q)
                sk_iteration<Real, Idx, ListT>(V, mask, r, c, lists + lo, nc, lists + n + lo, nr, G);
            if (leader) {
                n_full += nit;
                alg_bytes += (uint64_t)16 * (uint64_t)m_live * (uint64_t)nit;
            }
        } else if (use_local) {
            if (leader) {
                const int cr = mb[M_CNTR], cc = mb[M_CNTC];
                const uint64_t us = S.local_cap > 0 ? draw_u64(P.seed, traj, midx, (uint32_t)t, kLocalDraw) : 0;
                const int staged = local_repair<Real, Idx>(V, deg, mask, r, c, list_r, cr, list_c, cc, stamp, t + 1,
                                                           tmp_id, tmp_val, G.misc + M_TMP, lane, S.local_cap, us);
                ++n_loc;
                alg_bytes += (uint64_t)16 * (uint64_t)(staged + cr + cc);
            }
            gsync(G);
        }
    }
    if (leader && lane == 0) {
        if (!abandoned) P.log_x[gq] = (dead_step >= 0) ? -INFINITY : log_ratio(num, den);
        if (TRACE) P.dead_step[gq] = dead_step;
        unsigned long long* cnt = P.counters + kCounters * k;
        if (n_dm) atomicAdd(cnt + 0, (unsigned long long)n_dm);
        if (n_full) atomicAdd(cnt + 1, (unsigned long long)n_full);
        if (n_loc) atomicAdd(cnt + 2, (unsigned long long)n_loc);
        atomicAdd(cnt + 3, (unsigned long long)alg_bytes);
        if (mlp_rows) atomicAdd(cnt + 4, (unsigned long long)mlp_rows);
        atomicAdd(cnt + 5, (unsigned long long)(global_ns() - t_begin));
    }
    gsync(G);
}

// Whether the launch must start no further trajectory: its time budget is
// spent, or (checked by the CTA at chunk claims, `poll_cancel`) the host
// raised the context's cancel flag.  Sets the matching status bit.
__device__ __forceinline__ bool stop_starting(const TrajParams& P, bool poll_cancel)
{
    if (P.budget_ns) {
        const unsigned long long t0 = *reinterpret_cast<volatile unsigned long long*>(P.t_start);
        if (t0 && global_ns() - t0 > P.budget_ns) {
            atomicOr(P.status, ST_TIMEOUT);
            return true;
        }
    }
    if (poll_cancel && P.cancel && *P.cancel) {
        atomicOr(P.status, ST_CANCELLED);
        return true;
    }
    return false;
}

template <typename Real, typename Idx, bool TRACE, int MODE>
__device__ void run_chunk(const TrajParams& P, const Chunk& ch, const Plan& pl, const MV<Idx>& V, uint8_t* gstate,
                          int* ctr_traj, const DevModel* Ms)
{
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int gidx = warp / pl.g;
    if (gidx >= pl.groups) return;
    const int k = ch.k;
    const DevMatrix* Mp = P.mats + k;
    const int n = V.n;
    Grp G;
    G.g = pl.g;
    G.nthr = pl.g * 32;
    G.tid = tid - gidx * G.nthr;
    G.wig = G.tid >> 5;
    G.lane = lane;
    G.bar = 1 + gidx;
    G.gdm = pl.gstate && pl.g > 1;
    uint8_t* sbase = gstate + (size_t)gidx * pl.state_bytes;
    uint8_t* slot = P.slots + ((size_t)blockIdx.x * P.cta_warps + gidx) * P.slot.bytes;
    const TreeGeom T = tree_geom(n);
    // trajectory state: in shared memory, or (large n) in the group's slot
    uint8_t* base = pl.gstate ? slot + P.slot.state : sbase;
    uint16_t* deg = reinterpret_cast<uint16_t*>(base);
    size_t off = a16((size_t)((2 * n + 7) & ~7) * 2);
    uint32_t* tree = reinterpret_cast<uint32_t*>(base + off);
    off += a16((size_t)T.total * 4);
    Real* r_sm = nullptr;
    if (pl.rc_smem) {
        r_sm = reinterpret_cast<Real*>(base + off);
        off += 2 * a16((size_t)n * sizeof(Real));
    }
    uint8_t* lists = nullptr;  // [0, n): columns, [n, 2n): rows
    if (pl.lists) {
        lists = base + off;
        off += 2 * a16((size_t)n * (pl.gstate ? 4 : 2));
    }
    int* dm_sm = nullptr;      // the inner DM's workspace and edge mask (dm_smem plans)
    uint8_t* mask_sm = nullptr;
    if (pl.dm_smem && !pl.gstate) {
        dm_sm = reinterpret_cast<int*>(base + off);
        off += a16((size_t)dm_ws_ints(n) * 4);
        mask_sm = base + off;
        off += a16((size_t)Mp->m_a);
    }
    if (pl.gstate) off = 0;    // feature tile and control words stay in shared memory
    uint16_t* feat = nullptr;  // [32][kFS] bf16 feature tile of the learned proposal
    if (Ms) {
        feat = reinterpret_cast<uint16_t*>(sbase + off);
        off += 32 * kFS * 2;
    }
    G.misc = reinterpret_cast<int*>(sbase + off);
    for (;;) {
        if (G.wig == 0 && lane == 0)
            G.misc[M_TRAJ] = (P.budget_ns && stop_starting(P, false)) ? (int)ch.count : atomicAdd(ctr_traj, 1);
        gsync(G);
        const int q = G.misc[M_TRAJ];
        gsync(G);
        if (q >= (int)ch.count) break;
        const uint64_t local = ch.first + (uint64_t)q;
        const uint64_t gq = ch.slot0 + (uint64_t)q;
        if (pl.gstate)
            run_group<Real, Idx, TRACE, MODE, uint32_t>(P, Mp, V, k, gq, local, deg, tree, r_sm,
                                                        reinterpret_cast<uint32_t*>(lists), feat, Ms, slot, dm_sm, mask_sm, G);
        else
            run_group<Real, Idx, TRACE, MODE, uint16_t>(P, Mp, V, k, gq, local, deg, tree, r_sm,
                                                        reinterpret_cast<uint16_t*>(lists), feat, Ms, slot, dm_sm, mask_sm, G);
    }
}

#include "pm_pair.cuh"

// The persistent loop of a trajectory launch: CTAs claim chunks, stage the
// matrix when its plan says so, and run the chunk's trajectories.  PAIR_ONLY:
// every plan is a pair plan (the 768-thread kernel).
template <typename Real, bool TRACE, int MODE, bool PAIR_ONLY>
__device__ __forceinline__ void traj_body(const TrajParams& P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    int* cmisc = reinterpret_cast<int*>(smem);  // [0] chunk, [1] trajectory counter, [2] staged matrix
    const int tid = threadIdx.x;
    if (tid == 0) {
        cmisc[2] = -1;
        if (P.budget_ns) atomicCAS(P.t_start, 0ull, (unsigned long long)global_ns());  // the first CTA starts the clock
    }
    // the learned proposal's weights, staged once per CTA
    const DevModel* Ms = nullptr;
    int model_bytes = 0;
    if (MODE == 1) {
        model_bytes = (kModelInferBytes + 15) & ~15;
        const uint4* src = reinterpret_cast<const uint4*>(P.model);
        uint4* dst = reinterpret_cast<uint4*>(smem + kCtaMiscBytes);
        for (int q = tid; q < model_bytes / 16; q += blockDim.x) dst[q] = __ldg(src + q);
        Ms = reinterpret_cast<const DevModel*>(smem + kCtaMiscBytes);
    }
    for (;;) {
        __syncthreads();
        if (tid == 0) {
            cmisc[0] = stop_starting(P, true) ? P.n_chunks : atomicAdd(P.chunk_counter, 1);
            cmisc[1] = 0;
        }
        __syncthreads();
        const int ci = cmisc[0];
        if (ci >= P.n_chunks) break;
        const Chunk ch = P.chunks[ci];
        const Plan pl = P.plans[ch.k];
        const DevMatrix* Mp = P.mats + ch.k;
        const int n = Mp->n;
        uint8_t* mat = smem + kCtaMiscBytes + model_bytes;
        uint8_t* gstate = mat + pl.mat_bytes;
        if (pl.staged) {
            const int staged_k = cmisc[2];
            __syncthreads();
            const int m = Mp->m;
            int* s_rp = reinterpret_cast<int*>(mat);
            int* s_cp = reinterpret_cast<int*>(mat + a16((size_t)(n + 1) * 4));
            uint16_t* s_ci = reinterpret_cast<uint16_t*>(mat + 2 * a16((size_t)(n + 1) * 4));
            uint16_t* s_ri = reinterpret_cast<uint16_t*>(mat + 2 * a16((size_t)(n + 1) * 4) + a16((size_t)m * 2));
            int* s_ce = reinterpret_cast<int*>(mat + 2 * a16((size_t)(n + 1) * 4) + 2 * a16((size_t)m * 2));
            if (staged_k != ch.k) {
                for (int q = tid; q <= n; q += blockDim.x) { s_rp[q] = __ldg(Mp->rp + q); s_cp[q] = __ldg(Mp->cp + q); }
                for (int q = tid; q < m; q += blockDim.x) {
                    s_ci[q] = (uint16_t)__ldg(Mp->ci + q);
                    s_ri[q] = (uint16_t)__ldg(Mp->ri + q);
                }
                if (P.s.dm != DMP_NONE)
                    for (int q = tid; q < m; q += blockDim.x) s_ce[q] = __ldg(Mp->ce + q);
                if (tid == 0) cmisc[2] = ch.k;
            }
            __syncthreads();
            const MV<uint16_t> V = make_mv<uint16_t>(n, m, s_rp, s_cp, s_ci, s_ri, s_ce, Mp->rv, Mp->cv);
            if constexpr (PAIR_ONLY) {
                run_chunk_pair<Real, uint16_t, MODE>(P, ch, pl, V, gstate, cmisc + 1, Ms);
            } else {
                if constexpr (!TRACE && MODE != 2) {
                    if (pl.pair) {
                        run_chunk_pair<Real, uint16_t, MODE>(P, ch, pl, V, gstate, cmisc + 1, Ms);
                        continue;
                    }
                }
                run_chunk<Real, uint16_t, TRACE, MODE>(P, ch, pl, V, gstate, cmisc + 1, Ms);
            }
        } else {
            const MV<int> V = make_mv<int>(n, Mp->m, Mp->rp, Mp->cp, Mp->ci, Mp->ri, Mp->ce, Mp->rv, Mp->cv);
            if constexpr (PAIR_ONLY) {
                run_chunk_pair<Real, int, MODE>(P, ch, pl, V, gstate, cmisc + 1, Ms);
            } else {
                if constexpr (!TRACE && MODE != 2) {
                    if (pl.pair) {
                        run_chunk_pair<Real, int, MODE>(P, ch, pl, V, gstate, cmisc + 1, Ms);
                        continue;
                    }
                }
                run_chunk<Real, int, TRACE, MODE>(P, ch, pl, V, gstate, cmisc + 1, Ms);
            }
        }
    }
}

template <typename Real, bool TRACE, int MODE>
__global__ void __launch_bounds__(kCtaWarps * 32, 1) traj_kernel(TrajParams P)
{
    traj_body<Real, TRACE, MODE, false>(P);
}

template <typename Real>
__global__ void __launch_bounds__(kPairCtaWarps * 32, 1) traj_pair_kernel(TrajParams P)
{
    traj_body<Real, false, 0, true>(P);
}

// largest dynamic shared memory a launch of fn may request: the device's
// opt-in maximum less the kernel's static shared memory
int dyn_smem_cap(const void* fn)
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes a{};
    if (cudaFuncGetAttributes(&a, fn) != cudaSuccess) return 0;
    return v - (int)a.sharedSizeBytes;
}

template <typename Real, bool TRACE, int MODE>
cudaError_t launch_t(const TrajParams& p, int grid, int smem, cudaStream_t st)
{
    if constexpr (!TRACE && MODE == 0) {
        if (p.pair_kernel) {
            const int cap = dyn_smem_cap((const void*)traj_pair_kernel<Real>);
            cudaError_t e = cudaFuncSetAttribute(traj_pair_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 smem > cap ? smem : cap);
            if (e != cudaSuccess) return e;
            traj_pair_kernel<Real><<<grid, kPairCtaWarps * 32, smem, st>>>(p);
            return cudaGetLastError();
        }
    }
    // the attribute is a per-function cap shared by every launch and by the
    // kernel nodes of captured graphs: keep it at the device maximum so a
    // later, smaller launch never lowers it below a captured node's size
    const int cap = dyn_smem_cap((const void*)traj_kernel<Real, TRACE, MODE>);
    cudaError_t e = cudaFuncSetAttribute(traj_kernel<Real, TRACE, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem > cap ? smem : cap);
    if (e != cudaSuccess) return e;
    traj_kernel<Real, TRACE, MODE><<<grid, kCtaWarps * 32, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace

unsigned int traj_bounds_hits()
{
#ifdef PM_DEBUG
    unsigned int h = 0;
    const unsigned int z = 0;
    if (cudaMemcpyFromSymbol(&h, g_pm_bounds, sizeof(h)) != cudaSuccess) return ~0u;
    if (h && cudaMemcpyToSymbol(g_pm_bounds, &z, sizeof(z)) != cudaSuccess) return ~0u;
    return h;
#else
    return 0;
#endif
}

int traj_max_smem_bytes()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    return v;
}

const void* traj_kernel_entry(const TrajParams& p, bool trace)
{
    if (p.pair_kernel && !trace && !p.rec_feat && !p.model)
        return p.s.precision == 1 ? (const void*)traj_pair_kernel<double> : (const void*)traj_pair_kernel<float>;
    if (p.s.precision == 1)
        return trace ? (const void*)traj_kernel<double, true, 0> : (const void*)traj_kernel<double, false, 0>;
    if (p.model) return trace ? (const void*)traj_kernel<float, true, 1> : (const void*)traj_kernel<float, false, 1>;
    if (p.rec_feat) return (const void*)traj_kernel<float, false, 2>;
    return trace ? (const void*)traj_kernel<float, true, 0> : (const void*)traj_kernel<float, false, 0>;
}

cudaError_t launch_trajectories(const TrajParams& p, int grid, int smem, bool trace, cudaStream_t st)
{
    if (p.s.precision == 1) {
        if (p.model || p.rec_feat) return cudaErrorInvalidValue;  // learned / record are FP32-only
        return trace ? launch_t<double, true, 0>(p, grid, smem, st) : launch_t<double, false, 0>(p, grid, smem, st);
    }
    if (p.model) return trace ? launch_t<float, true, 1>(p, grid, smem, st) : launch_t<float, false, 1>(p, grid, smem, st);
    if (p.rec_feat) return launch_t<float, false, 2>(p, grid, smem, st);
    return trace ? launch_t<float, true, 0>(p, grid, smem, st) : launch_t<float, false, 0>(p, grid, smem, st);
}

}  // namespace pm
