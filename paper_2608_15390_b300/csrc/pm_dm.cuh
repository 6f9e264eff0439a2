// pm_dm.cuh -- support filtering by the Dulmage-Mendelsohn criterion
// (Sec. 2, "Support filtering with DM"): find a perfect matching M of the
// active part; orient M's edges row -> column and the others column -> row; a
// non-matching edge belongs to some perfect matching iff its two ends share a
// strongly connected component.  Single-thread version over global scratch:
// used once per matrix for the initial DM and by one lane per trajectory for
// the inner DM.
#pragma once
#include "pm_device.cuh"

namespace pm {

// workspace (ints): mr[n] mc[n] vis[n] cur[n] stk[n+1] idx[2n] low[2n]
// comp[2n] it[2n] onst[2n] cstk[2n+1] sstk[2n+1]
__host__ __device__ inline int dm_serial_ints(int n) { return 19 * n + 3; }

// Live must provide: bool row(int i), bool col(int j), bool edge(int e, int i, int j)
template <class Live, typename Idx>
__device__ bool dm_serial(int n, const int* rp, const Idx* ci, const int* cp, const Idx* ri,
                          const int* ce, const Live& live, uint8_t* mask, int* ws)
{
    int* mr = ws;
    int* mc = mr + n;
    int* vis = mc + n;
    int* cur = vis + n;
    int* stk = cur + n;
    int* idx = stk + n + 1;
    int* low = idx + 2 * n;
    int* comp = low + 2 * n;
    int* it = comp + 2 * n;
    int* onst = it + 2 * n;
    int* cstk = onst + 2 * n;
    int* sstk = cstk + 2 * n + 1;

    for (int i = 0; i < n; ++i) { mr[i] = -1; mc[i] = -1; vis[i] = -1; }
    // cheap greedy start, then one augmenting-path search per free row
    for (int i = 0; i < n; ++i) {
        if (!live.row(i)) continue;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            if (mc[j] < 0 && live.edge(e, i, j)) { mr[i] = j; mc[j] = i; break; }
        }
    }
    // Augmenting-path phases: within a phase the visited marks are shared by
    // all searches, so a phase costs O(m); a phase that augments nothing
    // proves the matching maximum (a failed search only marks columns from
    // which no free column is reachable).
    for (int phase = 0;; ++phase) {
        bool augmented = false, unmatched = false;
        for (int s = 0; s < n; ++s) {
            if (!live.row(s) || mr[s] >= 0) continue;
            unmatched = true;
            int top = 0;
            stk[0] = s;
            cur[s] = rp[s];
            while (top >= 0) {
                const int x = stk[top];
                if (cur[x] >= rp[x + 1]) { --top; continue; }
                const int e = cur[x]++;
                int j = ci[e];
                if (vis[j] == phase || !live.edge(e, x, j)) continue;
                vis[j] = phase;
                if (mc[j] < 0) {
                    for (int q = top; q >= 0; --q) {
                        const int row = stk[q];
                        const int prev = mr[row];
                        mr[row] = j;
                        mc[j] = row;
                        j = prev;
                    }
                    augmented = true;
                    break;
                }
                const int y = mc[j];
                stk[++top] = y;
                cur[y] = rp[y];
            }
        }
        if (!unmatched) break;
        if (!augmented) return false;
    }

    // strongly connected components (Tarjan, explicit stacks)
    const int V = 2 * n;
    for (int x = 0; x < V; ++x) { idx[x] = -1; onst[x] = 0; }
    int counter = 0, ncomp = 0, sp = 0;
    for (int s = 0; s < V; ++s) {
        const bool act = s < n ? live.row(s) : live.col(s - n);
        if (!act || idx[s] >= 0) continue;
        int ctop = 0;
        cstk[0] = s;
        it[s] = -1;
        idx[s] = low[s] = counter++;
        sstk[sp++] = s;
        onst[s] = 1;
        while (ctop >= 0) {
            const int x = cstk[ctop];
            int w = -1;
            if (x < n) {
                if (it[x] < 0) { it[x] = 0; w = n + mr[x]; }
            } else {
                const int j = x - n;
                int k = it[x] < 0 ? cp[j] : it[x] + 1;
                for (; k < cp[j + 1]; ++k) {
                    const int i = ri[k];
                    if (mr[i] != j && live.edge(ce[k], i, j)) break;
                }
                it[x] = k;
                if (k < cp[j + 1]) w = ri[k];
            }
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
                continue;
            }
            if (low[x] == idx[x]) {
                int y;
                do { y = sstk[--sp]; onst[y] = 0; comp[y] = ncomp; } while (y != x);
                ++ncomp;
            }
            if (--ctop >= 0) {
                const int par = cstk[ctop];
                if (low[x] < low[par]) low[par] = low[x];
            }
        }
    }
    for (int i = 0; i < n; ++i) {
        if (!live.row(i)) continue;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int j = ci[e];
            if (mr[i] != j && live.edge(e, i, j) && comp[i] != comp[n + j]) mask[e] = 0;
        }
    }
    return true;
}

}  // namespace pm
