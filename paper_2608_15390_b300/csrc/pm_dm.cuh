// pm_dm.cuh -- support filtering by the Dulmage-Mendelsohn criterion
// (Sec. 2, "Support filtering with DM"): find a perfect matching M of the
// active part; orient M's edges row -> column and the others column -> row; a
// non-matching edge belongs to some perfect matching iff its two ends share a
// strongly connected component.  One warp runs it (uniform control flow, ballots
// over adjacency chunks), once per matrix for the initial DM and by the leader
// warp of a trajectory for the inner DM.
#pragma once
#include "pm_device.cuh"

namespace pm {

// workspace (20 n + 3 of dm_ws_ints(n) = 21 n + 8 ints): mr[n] mc[n] vis[n]
// cur[n] stk[n+1] idx[2n] low[2n] comp[2n] it[2n] onst[2n] cstk[2n+1]
// sstk[2n+1] roots[2n]
struct DmWs {
    int *mr, *mc, *vis, *cur, *stk, *idx, *low, *comp, *it, *onst, *cstk, *sstk, *roots;
    __device__ DmWs(int* ws, int n)
    {
        mr = ws; mc = mr + n; vis = mc + n; cur = vis + n; stk = cur + n; idx = stk + n + 1; low = idx + 2 * n;
        comp = low + 2 * n; it = comp + 2 * n; onst = it + 2 * n; cstk = onst + 2 * n; sstk = cstk + 2 * n + 1;
        roots = sstk + 2 * n + 1;
    }
};



// Every lane follows the same (uniform) control flow and writes the same
// values; each search step examines up to 32 adjacency entries at once with a
// ballot and takes the first eligible entry in adjacency order.  Matching: a
// greedy start (or the repaired matching of the previous call), then
// augmenting-path phases whose searches share visited marks; free rows and
// unvisited vertices are found 32 at a time by ballots.
// Live must provide: bool row(int i), bool col(int j), bool edge(int e, int i, int j).
// repair: mr/mc already hold a matching of an earlier residual of the same
// matrix (the trajectory's previous DM call).  Pairs whose other end has been
// eliminated since are dropped and the search starts from that matching
// instead of the greedy one: after k eliminations at most k rows are free, so
// few augmenting searches remain.  The supported-edge set does not depend on
// which perfect matching the SCC step starts from, so the result is the same.
template <class Live, typename Idx>
__device__ bool dm_match_warp(int n, const int* rp, const Idx* ci, const Live& live, int* ws, int lane, bool repair)
{
    const DmWs W(ws, n);
    int *mr = W.mr, *mc = W.mc, *vis = W.vis, *cur = W.cur, *stk = W.stk;

    if (repair) {
        for (int i = lane; i < n; i += 32) {
            vis[i] = -1;
            if (live.row(i) && mr[i] >= 0 && !live.col(mr[i])) mr[i] = -1;
            if (live.col(i) && mc[i] >= 0 && !live.row(mc[i])) mc[i] = -1;
        }
    } else {
        for (int i = lane; i < n; i += 32) { mr[i] = -1; mc[i] = -1; vis[i] = -1; }
    }
    __syncwarp();
    // greedy start: each active row takes its first free live column; rows
    // with at most two entries go first (they have the fewest choices, so
    // matching them early leaves fewer rows for the augmenting phases)
    for (int it = 0; it < 2 * n && !repair; ++it) {
        const int i = it < n ? it : it - n;
        const bool short_row = rp[i + 1] - rp[i] <= 2;
        if (it < n ? !short_row : (short_row || mr[i] >= 0)) continue;
        if (!live.row(i)) continue;
        const int b = rp[i], en = rp[i + 1];
        for (int base = b; base < en; base += 32) {
            const int e = base + lane;
            bool ok = false;
            int j = 0;
            if (e < en) {
                j = ci[e];
                ok = mc[j] < 0 && live.edge(e, i, j);
            }
            const unsigned bal = __ballot_sync(kFull, ok);
            if (bal) {
                const int jj = __shfl_sync(kFull, j, __ffs(bal) - 1);
                mr[i] = jj;
                mc[jj] = i;
                __syncwarp();
                break;
            }
        }
    }
    // augmenting-path phases whose searches share visited marks (O(m) per
    // phase); a phase that augments nothing proves the matching maximum (a
    // failed search only marks columns from which no free column is reachable)
    for (int phase = 0;; ++phase) {
        bool augmented = false, unmatched = false;
        for (int s0 = 0; s0 < n; s0 += 32) {
            // the free active rows of this block of 32, in index order
            unsigned freeb = __ballot_sync(kFull, s0 + lane < n && live.row(s0 + lane) && mr[s0 + lane] < 0);
            while (freeb) {
                const int s = s0 + __ffs(freeb) - 1;
                freeb &= freeb - 1u;
                if (mr[s] >= 0) continue;  // matched by an earlier search of this block
                unmatched = true;
                int top = 0;
                stk[0] = s;
                cur[s] = rp[s];
                __syncwarp();
                while (top >= 0) {
                    const int x = stk[top];
                    const int en = rp[x + 1];
                    const int c0 = cur[x];
                    if (c0 >= en) { --top; continue; }
                    const int e = c0 + lane;
                    bool ok = false;
                    int j = 0;
                    if (e < en) {
                        j = ci[e];
                        ok = vis[j] != phase && live.edge(e, x, j);
                    }
                    const unsigned bal = __ballot_sync(kFull, ok);
                    if (!bal) {
                        cur[x] = c0 + 32;
                        __syncwarp();
                        continue;
                    }
                    const int l = __ffs(bal) - 1;
                    int jj = __shfl_sync(kFull, j, l);
                    cur[x] = c0 + l + 1;
                    vis[jj] = phase;
                    __syncwarp();
                    if (mc[jj] < 0) {
                        for (int q = top; q >= 0; --q) {
                            const int row = stk[q];
                            const int prev = mr[row];
                            __syncwarp();
                            mr[row] = jj;
                            mc[jj] = row;
                            __syncwarp();
                            jj = prev;
                        }
                        augmented = true;
                        break;
                    }
                    const int y = mc[jj];
                    stk[++top] = y;
                    cur[y] = rp[y];
                    __syncwarp();
                }
            }
        }
        if (!unmatched) break;
        if (!augmented) return false;
    }
    return true;
}

// Strongly connected components of the oriented residual (matching edges
// row -> column, the others column -> row) by Tarjan with explicit stacks,
// one warp; the next successor of a column is found by a ballot over its
// adjacency.  presolved: comp[x] in [0, 2n) marks a vertex whose component
// an earlier pass already found (a whole component of the graph, so the
// components of the other vertices are those of the graph without it); such
// vertices are neither visited nor followed, the new components get ids
// 2n + k, and the searches start from the nroots vertices of W.roots (the
// unsettled ones, whose idx = -1 and onst = 0 the caller set).  Otherwise
// every active vertex is visited and ids start at 0.
template <class Live, typename Idx>
__device__ void dm_tarjan_warp(int n, const int* cp, const Idx* ri, const int* ce, const Live& live, int* ws,
                               int lane, bool presolved, int nroots = 0)
{
    const DmWs W(ws, n);
    int *mr = W.mr, *idx = W.idx, *low = W.low, *comp = W.comp, *it = W.it, *onst = W.onst, *cstk = W.cstk,
        *sstk = W.sstk;
    const int V = 2 * n;
    auto solved = [&](int x) { return presolved && comp[x] >= 0 && comp[x] < V; };
    int* ib = W.vis;  // [2n] over vis and cur, which the matching no longer needs
    if (!presolved) {
        for (int x = lane; x < V; x += 32) { idx[x] = -1; onst[x] = 0; }
        __syncwarp();
    }
    int counter = 0, ncomp = presolved ? V : 0, sp = 0;
    const int nscan = presolved ? nroots : V;
    for (int s0 = 0; s0 < nscan; s0 += 32) {
      const int q = s0 + lane;
      const int sl = q < nscan ? (presolved ? W.roots[q] : q) : 0;
      unsigned todo = __ballot_sync(kFull, q < nscan && (sl < n ? live.row(sl) : live.col(sl - n)) && idx[sl] < 0 &&
                                               !solved(sl));
      while (todo) {
        const int s = __shfl_sync(kFull, sl, __ffs(todo) - 1);
        todo &= todo - 1u;
        if (idx[s] >= 0) continue;  // reached by an earlier search of this block
        int ctop = 0;
        cstk[0] = s;
        it[s] = -1;
        idx[s] = low[s] = counter++;
        sstk[sp++] = s;
        onst[s] = 1;
        __syncwarp();
        while (ctop >= 0) {
            const int x = cstk[ctop];
            int w = -1;
            if (x < n) {
                if (it[x] < 0) {
                    it[x] = 0;
                    w = n + mr[x];
                    if (solved(w)) w = -1;
                }
            } else {
                // the eligible entries of the chunk scanned last stay in ib[x]
                // (eligibility is fixed during the SCC step), so returning to
                // a column takes its next successor without re-reading the chunk
                const int j = x - n;
                const int en = cp[j + 1];
                const unsigned bits = it[x] < 0 ? 0u : (unsigned)ib[x];
                if (bits) {
                    w = ri[it[x] + __ffs(bits) - 1];
                    ib[x] = (int)(bits & (bits - 1u));
                } else {
                    int k = it[x] < 0 ? cp[j] : it[x] + 32;
                    bool found = false;
                    while (k < en) {
                        const int kk = k + lane;
                        bool ok = false;
                        int i = 0;
                        if (kk < en) {
                            i = ri[kk];
                            ok = mr[i] != j && live.edge(ce[kk], i, j) && !solved(i);
                        }
                        const unsigned bal = __ballot_sync(kFull, ok);
                        if (bal) {
                            w = __shfl_sync(kFull, i, __ffs(bal) - 1);
                            it[x] = k;
                            ib[x] = (int)(bal & (bal - 1u));
                            found = true;
                            break;
                        }
                        k += 32;
                    }
                    if (!found) {
                        it[x] = en;
                        ib[x] = 0;
                    }
                }
            }
            __syncwarp();
            if (w >= 0) {
                if (idx[w] < 0) {
                    idx[w] = low[w] = counter++;
                    sstk[sp++] = w;
                    onst[w] = 1;
                    it[w] = -1;
                    cstk[++ctop] = w;
                } else if (onst[w] && idx[w] < low[x]) {
                    low[x] = idx[w];
                }
                __syncwarp();
                continue;
            }
            if (low[x] == idx[x]) {
                int y;
                do {
                    y = sstk[--sp];
                    __syncwarp();
                    onst[y] = 0;
                    comp[y] = ncomp;
                    __syncwarp();
                } while (y != x);
                ++ncomp;
            }
            if (--ctop >= 0) {
                const int par = cstk[ctop];
                if (low[x] < low[par]) low[par] = low[x];
            }
            __syncwarp();
        }
      }
    }
    __syncwarp();
}

// Remove the unsupported edges: a live non-matching edge whose ends lie in
// different components (rows tid, tid + nthr, ...).
template <class Live, typename Idx>
__device__ void dm_mask_rows(int n, const int* rp, const Idx* ci, const Live& live, uint8_t* mask, int* ws, int tid,
                             int nthr)
{
    const DmWs W(ws, n);
    for (int i = tid; i < n; i += nthr) {
        if (!live.row(i)) continue;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            if (W.mr[i] != j && live.edge(e, i, j) && W.comp[i] != W.comp[n + j]) mask[e] = 0;
        }
    }
}

// The whole DM step on one warp: perfect matching, components, mask.
template <class Live, typename Idx>
__device__ bool dm_warp(int n, const int* rp, const Idx* ci, const int* cp, const Idx* ri, const int* ce,
                        const Live& live, uint8_t* mask, int* ws, int lane, bool repair = false)
{
    if (!dm_match_warp<Live, Idx>(n, rp, ci, live, ws, lane, repair)) return false;
    dm_tarjan_warp<Live, Idx>(n, cp, ri, ce, live, ws, lane, false);
    dm_mask_rows<Live, Idx>(n, rp, ci, live, mask, ws, lane, 32);
    __syncwarp();
    return true;
}

// Group-parallel first pass of the component step for large residuals (all
// nthr threads of a trajectory's group; sync() is the group barrier; sh: 8
// ints of the group's shared memory).  Leaves comp[x] = -1 for the active
// vertices it does not settle and, for the ones it does, an id in [0, 2n) of
// a whole component:
//   1. trimming: an undone vertex with no undone successor or no undone
//      predecessor lies on no cycle of the undone vertices, so it is a
//      component of its own (two passes: each costs a sweep over the
//      residual, and chains that would need more passes are left to the
//      searches and Tarjan, which settle them as well);
//   2. rounds of one forward and one backward breadth-first search over the
//      undone vertices from a pivot p, the undone vertex with the longest
//      adjacency list (ties: the smallest id; a long list makes p likely to
//      sit in the giant component): their intersection is p's component.
//      Rounds repeat, with new pivots, while more than max(256, 2n / 64)
//      vertices are undone, at most 8 times.
// What is left goes to W.roots (with idx = -1, onst = 0), and its count is
// returned, for dm_tarjan_warp(presolved = true).  Every loop is bounded: two
// trimming passes, at most 8 rounds, and a search level adds at least one
// new vertex, so at most 2n levels per search.
template <class Live, typename Idx, class Sync>
__device__ int dm_scc_group_prepass(int n, const int* rp, const Idx* ci, const int* cp, const Idx* ri, const int* ce,
                                     const Live& live, int* ws, int tid, int nthr, int* sh, Sync sync)
{
    const DmWs W(ws, n);
    int *mr = W.mr, *mc = W.mc, *comp = W.comp;
    int* fw = W.idx;   // reached by the forward search
    int* bw = W.low;   // reached by the backward search
    int* qa = W.cstk;  // frontiers (2n + 1 ints each)
    int* qb = W.sstk;
    const int V = 2 * n;
    auto active = [&](int x) { return x < n ? live.row(x) : live.col(x - n); };
    for (int x = tid; x < V; x += nthr) {
        comp[x] = active(x) ? -1 : -2;
        fw[x] = 0;
        bw[x] = 0;
    }
    if (tid == 0) { sh[0] = 0; sh[1] = 0; sh[2] = 0x7FFFFFFF; }
    sync();
    // 1. trimming
    for (int pass = 0; pass < 2; ++pass) {
        int* flag = sh + (pass & 1);
        for (int x = tid; x < V; x += nthr) {
            if (comp[x] != -1) continue;
            bool has_out = false, has_in = false;
            if (x < n) {  // row x: out = its matched column; in = its other live columns
                has_out = comp[n + mr[x]] == -1;
                for (int e = rp[x]; e < rp[x + 1] && !has_in; ++e) {
                    const int j = ci[e];
                    has_in = j != mr[x] && live.edge(e, x, j) && comp[n + j] == -1;
                }
            } else {      // column j: in = its matched row; out = its other live rows
                const int j = x - n;
                has_in = comp[mc[j]] == -1;
                for (int k = cp[j]; k < cp[j + 1] && !has_out; ++k) {
                    const int i = ri[k];
                    has_out = i != mc[j] && live.edge(ce[k], i, j) && comp[i] == -1;
                }
            }
            if (!has_out || !has_in) {
                comp[x] = x;
                *flag = 1;
            }
        }
        sync();
        const bool changed = *flag != 0;
        if (tid == 0) sh[(pass + 1) & 1] = 0;  // the next pass's flag (last read two barriers ago)
        sync();
        if (!changed) break;
    }
    // 2. forward-backward rounds; pivot key: list length (capped at 511) over
    // 23 bits of (2^23 - 1 - id), so the largest key is the longest list with
    // the smallest id (2n < 2^23)
    const unsigned kIdMask = (1u << 23) - 1u;
    for (int round = 1; round <= 8; ++round) {
    if (tid == 0) { sh[2] = 0; sh[3] = 0; }
    sync();
    for (int x = tid; x < V; x += nthr) {
        if (comp[x] != -1) continue;
        const int len = x < n ? rp[x + 1] - rp[x] : cp[x - n + 1] - cp[x - n];
        const unsigned key = ((unsigned)min(len, 511) << 23) | (kIdMask - (unsigned)x);
        atomicMax(reinterpret_cast<unsigned*>(sh + 2), key);
    }
    sync();
    const unsigned pk = (unsigned)sh[2];
    if (pk == 0) break;  // every vertex settled
    const int p = (int)(kIdMask - (pk & kIdMask));
    for (int dir = 0; dir < 2; ++dir) {  // 0: forward (successors), 1: backward (predecessors)
        int* mark = dir == 0 ? fw : bw;
        if (tid == 0) {
            mark[p] = round;
            qa[0] = p;
            sh[4] = 1;  // frontier size
            sh[5] = 0;
            sh[6] = 0;
        }
        sync();
        int* cur = qa;
        int* nxt = qb;
        for (int level = 0; level < V; ++level) {
            const int cnt = sh[4 + (level & 1)];
            int* ncnt = sh + 4 + ((level + 1) & 1);
            for (int q = tid; q < cnt; q += nthr) {
                const int x = cur[q];
                auto visit = [&](int y) {
                    if (comp[y] == -1 && atomicExch(&mark[y], round) != round) nxt[atomicAdd(ncnt, 1)] = y;
                };
                if (x < n) {
                    if (dir == 0) {
                        visit(n + mr[x]);
                    } else {
                        for (int e = rp[x]; e < rp[x + 1]; ++e) {
                            const int j = ci[e];
                            if (j != mr[x] && live.edge(e, x, j)) visit(n + j);
                        }
                    }
                } else {
                    const int j = x - n;
                    if (dir == 1) {
                        visit(mc[j]);
                    } else {
                        for (int k = cp[j]; k < cp[j + 1]; ++k) {
                            const int i = ri[k];
                            if (i != mc[j] && live.edge(ce[k], i, j)) visit(i);
                        }
                    }
                }
            }
            sync();
            const int next = *ncnt;
            if (tid == 0) sh[4 + (level & 1)] = 0;  // free the slot read at this level
            int* tq = cur;
            cur = nxt;
            nxt = tq;
            sync();
            if (next == 0) break;
        }
    }
    for (int x = tid; x < V; x += nthr) {
        if (comp[x] != -1) continue;
        if (fw[x] == round && bw[x] == round) comp[x] = p;
        else atomicAdd(sh + 3, 1);  // still undone
    }
    sync();
    const int left = sh[3];
    sync();
    if (left <= max(256, V / 64)) break;
    }
    // the unsettled vertices, for Tarjan
    if (tid == 0) sh[7] = 0;
    sync();
    for (int x = tid; x < V; x += nthr) {
        if (comp[x] != -1) continue;
        W.roots[atomicAdd(sh + 7, 1)] = x;
        W.idx[x] = -1;
        W.onst[x] = 0;
    }
    sync();
    const int nroots = sh[7];
    sync();
    return nroots;
}

// Group-parallel repair of the kept perfect matching (all nthr threads of
// the group; sync() is the group barrier; sh: 8 ints of shared memory): pairs
// whose other end was eliminated are dropped, then every free active row gets
// an augmenting path by a breadth-first alternating search (rows -> live
// columns; a matched column leads on to its row) until a free column is
// reached, and thread 0 flips the path.  Returns false if some free row has
// no augmenting path (the residual has no perfect matching).  Bounded: each
// search level claims at least one new column.
template <class Live, typename Idx, class Sync>
__device__ bool dm_repair_group(int n, const int* rp, const Idx* ci, const Live& live, int* ws, int tid, int nthr,
                                int* sh, Sync sync)
{
    const DmWs W(ws, n);
    int *mr = W.mr, *mc = W.mc, *seen = W.vis, *par = W.cur, *freer = W.stk;
    int* qa = W.idx;  // row frontiers (2n ints each; at most n rows)
    int* qb = W.low;
    if (tid == 0) sh[0] = 0;
    sync();
    for (int i = tid; i < n; i += nthr) {
        if (live.row(i) && mr[i] >= 0 && !live.col(mr[i])) mr[i] = -1;
        if (live.col(i) && mc[i] >= 0 && !live.row(mc[i])) mc[i] = -1;
        seen[i] = 0;
    }
    sync();
    for (int i = tid; i < n; i += nthr)
        if (live.row(i) && mr[i] < 0) freer[atomicAdd(sh, 1)] = i;
    sync();
    const int nfree = sh[0];
    sync();
    for (int f = 0; f < nfree; ++f) {
        const int s = freer[f];
        const int stamp = f + 1;
        if (tid == 0) {
            qa[0] = s;
            sh[1] = -1;  // the free column found
            sh[2] = 1;   // frontier sizes (two slots)
            sh[3] = 0;
        }
        sync();
        int* cur = qa;
        int* nxt = qb;
        int found = -1;
        for (int level = 0; level < n; ++level) {
            const int cnt = sh[2 + (level & 1)];
            int* ncnt = sh + 2 + ((level + 1) & 1);
            for (int q = tid; q < cnt; q += nthr) {
                const int x = cur[q];
                for (int e = rp[x]; e < rp[x + 1]; ++e) {
                    const int j = ci[e];
                    if (!live.edge(e, x, j) || atomicExch(&seen[j], stamp) == stamp) continue;
                    par[j] = x;
                    if (mc[j] < 0) atomicCAS(sh + 1, -1, j);
                    else nxt[atomicAdd(ncnt, 1)] = mc[j];
                }
            }
            sync();
            found = sh[1];
            const int next = *ncnt;
            if (tid == 0) sh[2 + (level & 1)] = 0;
            int* tq = cur;
            cur = nxt;
            nxt = tq;
            sync();
            if (found >= 0 || next == 0) break;
        }
        if (found < 0) return false;
        if (tid == 0) {  // flip the alternating path ending at the free column
            int j = found;
            for (int guard = 0; guard <= n; ++guard) {
                const int i = par[j];
                const int nj = mr[i];
                mr[i] = j;
                mc[j] = i;
                if (i == s) break;
                j = nj;
            }
        }
        sync();
    }
    return true;
}

}  // namespace pm
