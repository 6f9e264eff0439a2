/*
 * pm_oracle.c -- plain, slow CPU oracle for the adaptive sequential-importance
 * permanent estimator ("The Quick and the Dead", Elbek et al.).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header or
 * table with the CUDA library; it is written from the paper's text:
 *
 *   per(A)                     Eq. 1 (definition), Ryser's formula (Sec. 2)
 *   one trajectory             Algorithm 2 (generic estimator) with the
 *                              vertex rules of Sec. 3.2 (two-sided minimum
 *                              degree) and Algorithm 1 (fixed row order)
 *   proposal / correction      Eq. 3 and the correction line of Algorithm 2
 *   SK iteration               Sec. 3.3 (column update, then row update)
 *   Local repair               Eq. 5 and the R_loc / C_loc sets of Sec. 3.3
 *   DM support filtering       Sec. 2 ("Support filtering with DM")
 *   DM policies                Sec. 3.3 (All, Thrs, Trck)
 *   statistics                 Sec. 2 (ESS, p_match), Sec. 3.2 (relative
 *                              spread), Sec. 4 "Metrics" (RSE, s_X with M-1)
 *
 * Readings where the paper is silent:
 *   R1 MD ties: the active vertex of smallest (live degree, unified id) where
 *      row i has id i and column j has id n+j.
 *   R2 the proposal of Eq. 3 is realised with integer weights
 *      w = max(1, floor((s/s_max) * 2^k)), k = 40 - bitlen(deg); the draw is
 *      exact-uniform on [0, W) from Philox4x32-10 (Lemire's multiply-shift
 *      with rejection); the correction uses the realised probability w/W.
 *   R3 SK/local sums run in adjacency (index) order; a vertex with no live
 *      edge keeps its old scale.
 *   R4 Adaptive runs max(0, ceil((1 - z) K)) sweeps.
 *   R5 FP32-proposal mode rounds every scaling / proposal operation to
 *      binary32 (computed in binary64 and rounded: for +,-,*,/ this equals
 *      direct binary32 arithmetic because 53 >= 2*24+2); log-weights and
 *      statistics are binary64.
 *
 * Learned proposal (an extension with no counterpart in the paper): per-edge
 * features, an 8-64-64-1 tanh-GELU network in FP64 (optionally rounding its
 * inputs and hidden activations to bfloat16), its own binary32 exponent of
 * the score, recording of (features, SK target) pairs grouped by step, and the
 * training losses with their gradients by back-propagation: the mean squared
 * error and the per-step centred squared error (the proposal of Eq. 3 only
 * sees a step's logits up to a common offset).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -pthread -lm
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as    */
/* easy as 1, 2, 3", SC'11): 10 rounds of the 4x32 S-box with Weyl key bumps. */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The a-th 64-bit draw of (trajectory, matrix, step): counter
 * (traj lo32, traj hi16 | matrix << 16, step, a / 2), key (seed lo32, seed hi32);
 * even a takes words 0,1 and odd a takes words 2,3 of the block. */
uint64_t or_draw_u64(uint64_t seed, uint64_t traj, uint32_t matrix, uint32_t step, uint32_t a)
{
    uint32_t ctr[4] = { (uint32_t)traj, (uint32_t)((traj >> 32) & 0xFFFFu) | (matrix << 16),
                        step, a >> 1 };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t o[4];
    or_philox4x32_10(ctr, key, o);
    return (a & 1u) ? (((uint64_t)o[2] << 32) | o[3]) : (((uint64_t)o[0] << 32) | o[1]);
}

#define OR_MAX_ATTEMPTS 256
/* learned proposal: features, hidden width, parameter count */
#define OR_NF 8
#define OR_NH 64
#define OR_NPARAM (OR_NH * OR_NF + OR_NH + OR_NH * OR_NH + OR_NH + OR_NH + 1)

/* Uniform integer in [0, W) (W >= 1): multiply-shift with rejection (Lemire,
 * "Fast random integer generation in an interval", 2019).  Returns -1 if all
 * attempts were rejected (probability < 2^-6000 for W < 2^40). */
int64_t or_uniform_below(uint64_t W, uint64_t seed, uint64_t traj, uint32_t matrix, uint32_t step)
{
    uint64_t thresh = (0 - W) % W; /* 2^64 mod W */
    for (uint32_t a = 0; a < OR_MAX_ATTEMPTS; ++a) {
        unsigned __int128 p = (unsigned __int128)or_draw_u64(seed, traj, matrix, step, a) * W;
        if ((uint64_t)p >= thresh) return (int64_t)(uint64_t)(p >> 64);
    }
    return -1;
}

/* ------------------------------------------------------------------------- */
/* Exact permanents                                                           */
/* ------------------------------------------------------------------------- */

/* Ryser's inclusion-exclusion (Sec. 2): per(A) = (-1)^n sum_{S subset cols}
 * (-1)^{|S|} prod_i sum_{j in S} a_ij, for an integer matrix, exact in 128-bit
 * arithmetic.  Result written as (hi, lo) two's complement halves. */
void or_ryser_int(int n, const int64_t* a, uint64_t* out_hi, uint64_t* out_lo)
{
    /* subsets S visited in Gray-code order: step k flips column j = ctz(k), so
     * the row sums sum_{j in S} a_ij change by +-a_ij (O(n) per subset) */
    __int128 total = 0;
    int64_t rs[64] = {0};
    uint64_t S = 0;
    for (uint64_t k = 1; k < ((uint64_t)1 << n); ++k) {
        const int j = __builtin_ctzll(k);
        S ^= (uint64_t)1 << j;
        const int64_t sign = (S >> j & 1u) ? 1 : -1;
        __int128 prod = 1;
        for (int i = 0; i < n; ++i) {
            rs[i] += sign * a[(int64_t)i * n + j];
            prod *= rs[i];
        }
        int bits = __builtin_popcountll(S);
        if ((n - bits) & 1) total -= prod; else total += prod;
    }
    unsigned __int128 u = (unsigned __int128)total;
    *out_hi = (uint64_t)(u >> 64);
    *out_lo = (uint64_t)u;
}

/* Ryser for a real matrix in long double. */
long double or_ryser_real(int n, const double* a)
{
    long double total = 0;
    for (uint64_t S = 1; S < ((uint64_t)1 << n); ++S) {
        long double prod = 1;
        for (int i = 0; i < n; ++i) {
            long double rs = 0;
            for (int j = 0; j < n; ++j)
                if (S >> j & 1u) rs += a[(int64_t)i * n + j];
            prod *= rs;
        }
        int bits = __builtin_popcountll(S);
        if ((n - bits) & 1) total -= prod; else total += prod;
    }
    return total;
}

double or_ryser_real_d(int n, const double* a) { return (double)or_ryser_real(n, a); }

/* ------------------------------------------------------------------------- */
/* Matrix, schedule and per-matrix preprocessing                              */
/* ------------------------------------------------------------------------- */

enum { VR_MIN_DEGREE_2SIDED = 0, VR_ROW_ORDER = 1 };
enum { SK_NONE = 0, SK_FIXED = 1, SK_ADAPTIVE = 2, SK_LOCAL = 3 };
enum { DM_NONE = 0, DM_ALL = 1, DM_THRS = 2, DM_TRCK = 3 };
enum { PREC_FP32 = 0, PREC_FP64 = 1 };

typedef struct {
    int32_t vertex_rule, initial_dm, K0, K, sk, dm, precision;
    int32_t local_cap;  /* 0: the Local repair of Eq. 5; L > 0: its bounded-work variant */
    double theta;
} or_schedule;

typedef struct {
    int n;
    int64_t m;
    const int64_t* rp;  /* CSR row pointer [n+1] */
    const int32_t* ci;  /* CSR column indices [m] */
    const float* val;   /* [m] or NULL (0/1 matrix) */
    int64_t* cp;        /* CSC column pointer [n+1] */
    int32_t* ri;        /* CSC row indices [m] */
    int64_t* ce;        /* CSC entry -> CSR entry */
    or_schedule s;
    int fp32;
    uint8_t* mask0;     /* edges kept by the initial DM (1) */
    /* B^(0) = A after the initial DM, every trajectory's starting matrix:
     * its row lists as A's edge ids (b0re, pointers b0rp) and its column
     * lists as A's CSC positions (b0ck, pointers b0cp), in A's order */
    int64_t *b0rp, *b0re, *b0cp, *b0ck;
    double* r0;         /* outer scaling, float-valued in FP32 mode */
    double* c0;
    int ok;             /* initial DM found a perfect matching */
    int max_steps;      /* > 0: stop every trajectory after this many steps (prefix replay) */
} or_prep;

static double rnd(int fp32, double x) { return fp32 ? (double)(float)x : x; }

static double entry(const or_prep* P, int64_t e) { return P->val ? (double)P->val[e] : 1.0; }

/* Trajectory state.  deg[] holds live degrees of unified vertices (row i -> i,
 * column j -> n + j); act[] marks active vertices; mask[] marks edges not yet
 * removed by DM. */
typedef struct {
    const or_prep* P;
    uint8_t* act;
    int32_t* deg;
    uint8_t* mask;
    double* r;
    double* c;
    /* DM workspaces */
    int32_t *mr, *mc, *stk, *it, *idx, *low, *comp, *sstk, *vis;
    uint8_t* onst;
    /* local-repair workspaces */
    int32_t *stampr, *stampc, *listr, *listc;
    double *newr, *newc;
    int32_t stamp;
    /* candidate lists */
    int64_t* cand_e;
    int32_t* cand_p;
    uint64_t* w;
    int32_t *nbrR, *nbrC;
    float* recbuf;   /* recording scratch: n rows of 8 features, n targets, n indices */
} or_traj;

static int edge_live(const or_traj* T, int64_t e, int row, int col)
{
    const int n = T->P->n;
    return T->mask[e] && T->act[row] && T->act[n + col];
}

/* Live degree straight from the definition: number of live edges at v. */
static int32_t live_degree(const or_traj* T, int v)
{
    const or_prep* P = T->P;
    const int n = P->n;
    int32_t d = 0;
    if (v < n) {
        for (int64_t e = P->rp[v]; e < P->rp[v + 1]; ++e) d += edge_live(T, e, v, P->ci[e]);
    } else {
        int j = v - n;
        for (int64_t k = P->cp[j]; k < P->cp[j + 1]; ++k) d += edge_live(T, P->ce[k], P->ri[k], j);
    }
    return d;
}

static void recompute_degrees(or_traj* T)
{
    const int n = T->P->n;
    for (int v = 0; v < 2 * n; ++v) T->deg[v] = T->act[v] ? live_degree(T, v) : 0;
}

/* ---- DM (Sec. 2): maximum matching by augmenting paths, then SCCs of the
 * oriented graph (matched edges row->col, others col->row); a non-matching
 * live edge survives iff both ends share an SCC.  Returns 0 when the active
 * part has no perfect matching. ---- */

/* one augmenting-path search from free row s (iterative DFS over rows) */
static int augment(or_traj* T, int s, int32_t visit_mark)
{
    const or_prep* P = T->P;
    int top = 0;
    T->stk[top] = s;
    T->it[s] = (int32_t)P->rp[s] - 1;
    while (top >= 0) {
        int i = T->stk[top];
        int64_t e = ++T->it[i];
        if (e >= P->rp[i + 1]) { --top; continue; }
        int j = P->ci[e];
        if (!edge_live(T, e, i, j) || T->vis[j] == visit_mark) continue;
        T->vis[j] = visit_mark;
        if (T->mc[j] < 0) {
            /* flip the alternating path: stk[q] takes the column stk[q+1]
             * was matched to (stk[top] takes the free column j) */
            int col = j;
            for (int q = top; q >= 0; --q) {
                int row = T->stk[q];
                int prev = T->mr[row];
                T->mr[row] = col;
                T->mc[col] = row;
                col = prev;
            }
            return 1;
        }
        int nxt = T->mc[j];
        T->stk[++top] = nxt;
        T->it[nxt] = (int32_t)P->rp[nxt] - 1;
    }
    return 0;
}

static int dm_filter(or_traj* T)
{
    const or_prep* P = T->P;
    const int n = P->n;
    for (int i = 0; i < n; ++i) T->mr[i] = -1;
    for (int j = 0; j < n; ++j) { T->mc[j] = -1; T->vis[j] = -1; }
    int32_t mark = 0;
    for (int i = 0; i < n; ++i) {
        if (!T->act[i]) continue;
        if (!augment(T, i, mark++)) return 0;
    }
    /* Tarjan SCC over active unified vertices, iterative. */
    const int V = 2 * n;
    for (int v = 0; v < V; ++v) { T->idx[v] = -1; T->onst[v] = 0; }
    int32_t counter = 0, ncomp = 0, sp = 0;
    for (int s = 0; s < V; ++s) {
        if (!T->act[s] || T->idx[s] >= 0) continue;
        int top = 0;
        T->stk[0] = s;
        T->it[s] = -1;
        T->idx[s] = T->low[s] = counter++;
        T->sstk[sp++] = s; T->onst[s] = 1;
        while (top >= 0) {
            int v = T->stk[top];
            int w = -1;
            /* next successor of v */
            if (v < n) {
                if (T->it[v] < 0) { T->it[v] = 0; w = n + T->mr[v]; }
            } else {
                int j = v - n;
                for (;;) {
                    int64_t k = (T->it[v] < 0) ? P->cp[j] : (int64_t)T->it[v] + 1;
                    if (k >= P->cp[j + 1]) { T->it[v] = (int32_t)P->cp[j + 1]; break; }
                    T->it[v] = (int32_t)k;
                    int i = P->ri[k];
                    if (edge_live(T, P->ce[k], i, j) && T->mr[i] != j) { w = i; break; }
                }
            }
            if (w >= 0) {
                if (T->idx[w] < 0) {
                    T->idx[w] = T->low[w] = counter++;
                    T->sstk[sp++] = w; T->onst[w] = 1;
                    T->it[w] = -1;
                    T->stk[++top] = w;
                } else if (T->onst[w] && T->idx[w] < T->low[v]) {
                    T->low[v] = T->idx[w];
                }
                continue;
            }
            if (T->low[v] == T->idx[v]) {
                int x;
                do { x = T->sstk[--sp]; T->onst[x] = 0; T->comp[x] = ncomp; } while (x != v);
                ++ncomp;
            }
            --top;
            if (top >= 0) {
                int u = T->stk[top];
                if (T->low[v] < T->low[u]) T->low[u] = T->low[v];
            }
        }
    }
    for (int i = 0; i < n; ++i) {
        if (!T->act[i]) continue;
        for (int64_t e = P->rp[i]; e < P->rp[i + 1]; ++e) {
            int j = P->ci[e];
            if (!edge_live(T, e, i, j) || T->mr[i] == j) continue;
            if (T->comp[i] != T->comp[n + j]) T->mask[e] = 0;
        }
    }
    recompute_degrees(T);
    return 1;
}

/* ---- SK (Sec. 3.3): one iteration updates every active column from r, then
 * every active row from the new c. ---- */
static double col_sum(const or_traj* T, int j, const double* r)
{
    const or_prep* P = T->P;
    double s = 0;
    for (int64_t k = P->cp[j]; k < P->cp[j + 1]; ++k) {
        int i = P->ri[k];
        int64_t e = P->ce[k];
        if (!edge_live(T, e, i, j)) continue;
        s = rnd(P->fp32, s + rnd(P->fp32, entry(P, e) * r[i]));
    }
    return s;
}

static double row_sum(const or_traj* T, int i, const double* c)
{
    const or_prep* P = T->P;
    double s = 0;
    for (int64_t e = P->rp[i]; e < P->rp[i + 1]; ++e) {
        int j = P->ci[e];
        if (!edge_live(T, e, i, j)) continue;
        s = rnd(P->fp32, s + rnd(P->fp32, entry(P, e) * c[j]));
    }
    return s;
}

static void sk_sweep(or_traj* T)
{
    const or_prep* P = T->P;
    const int n = P->n;
    for (int j = 0; j < n; ++j) {
        if (!T->act[n + j] || T->deg[n + j] == 0) continue;
        T->c[j] = rnd(P->fp32, 1.0 / col_sum(T, j, T->r));
    }
    for (int i = 0; i < n; ++i) {
        if (!T->act[i] || T->deg[i] == 0) continue;
        T->r[i] = rnd(P->fp32, 1.0 / row_sum(T, i, T->c));
    }
}

/* ---- Bounded-work Local repair.  Sec. 3.3 leaves it to future work: cap
 * the incident edges examined and approximate the local normalisation sums
 * by sampling the neighbourhood.  This build's reading, for a cap L > 0, with
 * lists taken in B^(0) (A after the initial DM: the matrix every trajectory
 * starts from, whose later residuals only mark entries dead):
 *   - the two-hop expansion skips a vertex whose B^(0) list (live and dead
 *     entries) is longer than L: its neighbours keep their scales;
 *   - the sum of a vertex whose list is longer than L is estimated from a
 *     systematic sample of L list positions k_q = (o + q s) mod len,
 *     q = 0..L-1, s = floor(len / L), o = u mod len, u the step's sampling
 *     word (Philox draw 2048 of the trajectory's step): the terms of the
 *     live sampled entries summed in sample order, times deg / (their count);
 *     no live sample keeps the old scale.
 * Scales only shape the proposal, and the weight uses the realised q, so the
 * estimator stays unbiased whatever L. ---- */
#define OR_LOCAL_DRAW 2048u

static double sampled_row_sum(const or_traj* T, int i, const double* c, uint64_t u, int L, int* cnt)
{
    const or_prep* P = T->P;
    const int64_t b = P->b0rp[i], len = P->b0rp[i + 1] - b, s = len / L, o = (int64_t)(u % (uint64_t)len);
    double acc = 0;
    int k = 0;
    for (int q = 0; q < L; ++q) {
        const int64_t e = P->b0re[b + (o + (int64_t)q * s) % len];
        const int j = P->ci[e];
        if (!edge_live(T, e, i, j)) continue;
        acc = rnd(P->fp32, acc + rnd(P->fp32, entry(P, e) * c[j]));
        ++k;
    }
    *cnt = k;
    return acc;
}

static double sampled_col_sum(const or_traj* T, int j, const double* r, uint64_t u, int L, int* cnt)
{
    const or_prep* P = T->P;
    const int64_t b = P->b0cp[j], len = P->b0cp[j + 1] - b, s = len / L, o = (int64_t)(u % (uint64_t)len);
    double acc = 0;
    int k = 0;
    for (int q = 0; q < L; ++q) {
        const int64_t kk = P->b0ck[b + (o + (int64_t)q * s) % len];
        const int i = P->ri[kk];
        const int64_t e = P->ce[kk];
        if (!edge_live(T, e, i, j)) continue;
        acc = rnd(P->fp32, acc + rnd(P->fp32, entry(P, e) * r[i]));
        ++k;
    }
    *cnt = k;
    return acc;
}

/* new scale of a vertex from its (possibly sampled) sum: 1 / (sum deg / cnt) */
static double scale_from_sample(const or_prep* P, double old, double sum, int deg, int cnt)
{
    if (cnt == 0) return old;
    const double est = rnd(P->fp32, rnd(P->fp32, sum * (double)deg) / (double)cnt);
    return rnd(P->fp32, 1.0 / est);
}

/* ---- Local repair (Eq. 5).  nR/nC: N_t(C)\{R} (rows) and N_t(R)\{C}
 * (columns), collected before elimination. R_loc = nR U N_{t+1}(nC),
 * C_loc = nC U N_{t+1}(nR); new values use only the old vectors and are
 * committed together.  cap L > 0: the bounded-work variant above, u the
 * step's sampling word. ---- */
static void local_repair(or_traj* T, const int32_t* nR, int cntR, const int32_t* nC, int cntC, int L,
                         uint64_t u)
{
    const or_prep* P = T->P;
    const int n = P->n;
    int32_t st = ++T->stamp;
    int lr = 0, lc = 0;
#define ADD_R(i) do { if (T->stampr[i] != st) { T->stampr[i] = st; T->listr[lr++] = (i); } } while (0)
#define ADD_C(j) do { if (T->stampc[j] != st) { T->stampc[j] = st; T->listc[lc++] = (j); } } while (0)
    for (int q = 0; q < cntR; ++q) ADD_R(nR[q]);
    for (int q = 0; q < cntC; ++q) ADD_C(nC[q]);
    for (int q = 0; q < cntC; ++q) { /* child neighbours of the columns in nC */
        int j = nC[q];
        if (L > 0 && P->b0cp[j + 1] - P->b0cp[j] > L) continue;
        for (int64_t k = P->cp[j]; k < P->cp[j + 1]; ++k)
            if (edge_live(T, P->ce[k], P->ri[k], j)) ADD_R(P->ri[k]);
    }
    for (int q = 0; q < cntR; ++q) { /* child neighbours of the rows in nR */
        int i = nR[q];
        if (L > 0 && P->b0rp[i + 1] - P->b0rp[i] > L) continue;
        for (int64_t e = P->rp[i]; e < P->rp[i + 1]; ++e)
            if (edge_live(T, e, i, P->ci[e])) ADD_C(P->ci[e]);
    }
#undef ADD_R
#undef ADD_C
    for (int q = 0; q < lr; ++q) {
        int i = T->listr[q];
        if (T->deg[i] == 0) {
            T->newr[q] = T->r[i];
        } else if (L > 0 && P->b0rp[i + 1] - P->b0rp[i] > L) {
            int cnt;
            const double sm = sampled_row_sum(T, i, T->c, u, L, &cnt);
            T->newr[q] = scale_from_sample(P, T->r[i], sm, T->deg[i], cnt);
        } else {
            T->newr[q] = rnd(P->fp32, 1.0 / row_sum(T, i, T->c));
        }
    }
    for (int q = 0; q < lc; ++q) {
        int j = T->listc[q];
        if (T->deg[n + j] == 0) {
            T->newc[q] = T->c[j];
        } else if (L > 0 && P->b0cp[j + 1] - P->b0cp[j] > L) {
            int cnt;
            const double sm = sampled_col_sum(T, j, T->r, u, L, &cnt);
            T->newc[q] = scale_from_sample(P, T->c[j], sm, T->deg[n + j], cnt);
        } else {
            T->newc[q] = rnd(P->fp32, 1.0 / col_sum(T, j, T->r));
        }
    }
    for (int q = 0; q < lr; ++q) T->r[T->listr[q]] = T->newr[q];
    for (int q = 0; q < lc; ++q) T->c[T->listc[q]] = T->newc[q];
}

/* ------------------------------------------------------------------------- */

static void* xcalloc(size_t n, size_t sz) { void* p = calloc(n ? n : 1, sz); return p; }

static or_traj* traj_alloc(const or_prep* P)
{
    const int n = P->n;
    or_traj* T = (or_traj*)xcalloc(1, sizeof(or_traj));
    T->P = P;
    T->act = (uint8_t*)xcalloc(2 * n, 1);
    T->deg = (int32_t*)xcalloc(2 * n, 4);
    T->mask = (uint8_t*)xcalloc(P->m, 1);
    T->r = (double*)xcalloc(n, 8);
    T->c = (double*)xcalloc(n, 8);
    T->mr = (int32_t*)xcalloc(n, 4);
    T->mc = (int32_t*)xcalloc(n, 4);
    T->vis = (int32_t*)xcalloc(n, 4);
    T->stk = (int32_t*)xcalloc(2 * n + 1, 4);
    T->it = (int32_t*)xcalloc(2 * n, 4);
    T->idx = (int32_t*)xcalloc(2 * n, 4);
    T->low = (int32_t*)xcalloc(2 * n, 4);
    T->comp = (int32_t*)xcalloc(2 * n, 4);
    T->sstk = (int32_t*)xcalloc(2 * n + 1, 4);
    T->onst = (uint8_t*)xcalloc(2 * n, 1);
    T->stampr = (int32_t*)xcalloc(n, 4);
    T->stampc = (int32_t*)xcalloc(n, 4);
    T->listr = (int32_t*)xcalloc(n, 4);
    T->listc = (int32_t*)xcalloc(n, 4);
    T->newr = (double*)xcalloc(n, 8);
    T->newc = (double*)xcalloc(n, 8);
    T->cand_e = (int64_t*)xcalloc(n, 8);
    T->cand_p = (int32_t*)xcalloc(n, 4);
    T->w = (uint64_t*)xcalloc(n, 8);
    T->nbrR = (int32_t*)xcalloc(n, 4);
    T->nbrC = (int32_t*)xcalloc(n, 4);
    T->recbuf = (float*)xcalloc((size_t)n * (OR_NF + 2), 4);
    return T;
}

static void traj_free(or_traj* T)
{
    if (!T) return;
    void* ptrs[] = { T->act, T->deg, T->mask, T->r, T->c, T->mr, T->mc, T->vis, T->stk, T->it,
                     T->idx, T->low, T->comp, T->sstk, T->onst, T->stampr, T->stampc, T->listr,
                     T->listc, T->newr, T->newc, T->cand_e, T->cand_p, T->w, T->nbrR, T->nbrC, T->recbuf };
    for (size_t q = 0; q < sizeof(ptrs) / sizeof(ptrs[0]); ++q) free(ptrs[q]);
    free(T);
}

/* Preprocessing of Algorithm 2: InitialDM, r = c = 1, K0 SK iterations. */
or_prep* or_prepare(int n, int64_t m, const int64_t* rp, const int32_t* ci, const float* val,
                    const or_schedule* s)
{
    or_prep* P = (or_prep*)xcalloc(1, sizeof(or_prep));
    P->n = n; P->m = m; P->rp = rp; P->ci = ci; P->val = val; P->s = *s;
    P->fp32 = (s->precision == PREC_FP32);
    P->cp = (int64_t*)xcalloc(n + 1, 8);
    P->ri = (int32_t*)xcalloc(m, 4);
    P->ce = (int64_t*)xcalloc(m, 8);
    for (int64_t e = 0; e < m; ++e) P->cp[ci[e] + 1]++;
    for (int j = 0; j < n; ++j) P->cp[j + 1] += P->cp[j];
    int64_t* fill = (int64_t*)xcalloc(n, 8);
    for (int i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            int j = ci[e];
            int64_t k = P->cp[j] + fill[j]++;
            P->ri[k] = i;
            P->ce[k] = e;
        }
    free(fill);
    P->mask0 = (uint8_t*)xcalloc(m, 1);
    P->r0 = (double*)xcalloc(n, 8);
    P->c0 = (double*)xcalloc(n, 8);
    or_traj* T = traj_alloc(P);
    memset(T->act, 1, 2 * (size_t)n);
    memset(T->mask, 1, (size_t)m);
    P->ok = 1;
    recompute_degrees(T);
    if (s->initial_dm) P->ok = dm_filter(T);
    for (int v = 0; v < n; ++v) { T->r[v] = 1.0; T->c[v] = 1.0; }
    if (P->ok)
        for (int k = 0; k < s->K0; ++k) sk_sweep(T);
    memcpy(P->mask0, T->mask, (size_t)m);
    P->b0rp = (int64_t*)xcalloc(n + 1, 8);
    P->b0cp = (int64_t*)xcalloc(n + 1, 8);
    P->b0re = (int64_t*)xcalloc(m, 8);
    P->b0ck = (int64_t*)xcalloc(m, 8);
    for (int i = 0; i < n; ++i) {
        P->b0rp[i + 1] = P->b0rp[i];
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (P->mask0[e]) P->b0re[P->b0rp[i + 1]++] = e;
    }
    for (int j = 0; j < n; ++j) {
        P->b0cp[j + 1] = P->b0cp[j];
        for (int64_t k = P->cp[j]; k < P->cp[j + 1]; ++k)
            if (P->mask0[P->ce[k]]) P->b0ck[P->b0cp[j + 1]++] = k;
    }
    memcpy(P->r0, T->r, (size_t)n * 8);
    memcpy(P->c0, T->c, (size_t)n * 8);
    traj_free(T);
    return P;
}

void or_prep_free(or_prep* P)
{
    if (!P) return;
    free(P->cp); free(P->ri); free(P->ce); free(P->mask0); free(P->r0); free(P->c0);
    free(P->b0rp); free(P->b0re); free(P->b0cp); free(P->b0ck);
    free(P);
}

int or_prep_ok(const or_prep* P) { return P->ok; }
void or_prep_set_max_steps(or_prep* P, int max_steps) { P->max_steps = max_steps; }
void or_prep_scaling(const or_prep* P, double* r, double* c)
{
    memcpy(r, P->r0, (size_t)P->n * 8);
    memcpy(c, P->c0, (size_t)P->n * 8);
}
void or_prep_mask(const or_prep* P, uint8_t* mask) { memcpy(mask, P->mask0, (size_t)P->m); }

/* ------------------------------------------------------------------------- */
/* One trajectory of Algorithm 2                                              */
/* ------------------------------------------------------------------------- */

typedef struct {
    double log_x;        /* ln X, -INFINITY if the trajectory died */
    int32_t dead_step;   /* step at which it died, -1 if it completed */
    int32_t dead_reason; /* 0 none, 1 empty neighbourhood, 2 InnerDM found no matching, 3 rng */
    int32_t n_dm, n_full_sk, n_local_sk, pad;
} or_traj_result;

/* forced-choice interface for exhaustive enumeration: when forced != NULL the
 * t-th step takes candidate forced[t] instead of a Philox draw; when t reaches
 * n_forced the function stops and reports the candidate weights (need_choice). */
/* learned-proposal hooks (an extension; the paper has no learned
 * proposal): ext_logits[t * lstride + q] is the logit of the q-th live
 * candidate at step t (lstride >= the largest candidate count; a step with
 * more candidates cannot be replayed and ends the trajectory with
 * dead_reason 4); record_* collect (features, target) pairs of the SK
 * estimator. */
typedef struct {
    const double* model;       /* [4801] network parameters, or NULL */
    const float* ext_logits;   /* [n][lstride] or NULL */
    int32_t lstride;           /* row length of ext_logits and model_logits_out */
    float* rec_feat;           /* [cap][8] or NULL */
    float* rec_target;         /* [cap] */
    uint64_t* rec_key;         /* [cap]: traj << 28 | t << 14 | q */
    uint32_t* rec_group;       /* [cap] or NULL: index within the step's pairs << 16 | their count */
    int64_t rec_cap, rec_n;
    int rec_full;              /* a step's pairs no longer fit: recording has stopped */
    float* model_logits_out;   /* [n][lstride] or NULL: the network's own logits along the path */
} or_learn;

typedef struct {
    const int32_t* forced;
    int32_t n_forced;
    int32_t need_choice;   /* out: 1 if stopped for a choice */
    int32_t n_cand;        /* out: candidate count at that step */
    uint64_t* w_out;       /* out: candidate weights (caller-sized >= n) */
    uint64_t W_out;        /* out */
    double* logx_prefix;   /* out: ln X so far */
} or_forced;

static int bitlen32(uint32_t x) { return x ? 32 - __builtin_clz(x) : 0; }

/* Score of the learned proposal: e^x for x clamped to [-20, 20] (NaN -> -20),
 * computed as 2^(x log2 e) with a degree-7 Taylor polynomial of
 * 2^f = e^(f ln 2) on |f| <= 1/2.  Every step is a correctly rounded binary32
 * operation (no contraction); the coefficients are (ln 2)^k / k! rounded to
 * binary32, and log2 e rounded to binary32. */
float or_exp_score(float x)
{
    static const float C[8] = { 1.0f, 0x1.62e430p-1f, 0x1.ebfbe0p-3f, 0x1.c6b08ep-5f,
                                0x1.3b2ab6p-7f, 0x1.5d87fep-10f, 0x1.430912p-13f, 0x1.ffcbfcp-17f };
    if (!(x >= -20.0f)) x = -20.0f;
    if (x > 20.0f) x = 20.0f;
    const float y = x * 0x1.715476p+0f;
    const float nn = nearbyintf(y);
    const float f = y - nn;
    float p = C[7];
    for (int k = 6; k >= 0; --k) p = p * f + C[k];
    return ldexpf(p, (int)nn);
}


/* Per-edge features of candidate (v, l) at step t (residual degrees,
 * neighbour-degree sums, depth fraction, current scale): log1p deg(v), log1p deg(l), log1p of the degree sum over v's
 * live candidates, log1p of the degree sum over l's live neighbours, t / n,
 * ln of the outer scale of v and of l (r for rows, c for columns), ln B_vl. */
static void edge_features(const or_traj* T, int t, int v, int l_unified, int64_t e, double sum_v, float* f)
{
    const or_prep* P = T->P;
    const int n = P->n;
    double sum_l = 0;
    if (l_unified < n) {
        for (int64_t k = P->rp[l_unified]; k < P->rp[l_unified + 1]; ++k)
            if (edge_live(T, k, l_unified, P->ci[k])) sum_l += T->deg[n + P->ci[k]];
    } else {
        const int j = l_unified - n;
        for (int64_t k = P->cp[j]; k < P->cp[j + 1]; ++k)
            if (edge_live(T, P->ce[k], P->ri[k], j)) sum_l += T->deg[P->ri[k]];
    }
    const double sv = v < n ? P->r0[v] : P->c0[v - n];
    const double sl = l_unified < n ? P->r0[l_unified] : P->c0[l_unified - n];
    f[0] = (float)log1p((double)T->deg[v]);
    f[1] = (float)log1p((double)T->deg[l_unified]);
    f[2] = (float)log1p(sum_v);
    f[3] = (float)log1p(sum_l);
    f[4] = (float)((double)t / (double)n);
    f[5] = (float)log(sv);
    f[6] = (float)log(sl);
    f[7] = (float)log(entry(P, e));
}

/* MLP 8 -> 64 -> 64 -> 1 with GELU in its tanh form,
 * g(x) = x/2 (1 + tanh(c (x + a x^3))), c = sqrt(2/pi), a = 0.044715;
 * parameters laid out as W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3.
 * round_act rounds the hidden activations to bfloat16 (round to nearest
 * even) as tensor-core inference does. */
static const double GELU_C = 0.79788456080286535588, GELU_A = 0.044715;
static double gelu(double x) { return 0.5 * x * (1.0 + tanh(GELU_C * (x + GELU_A * x * x * x))); }
static double gelu_d(double x)
{
    const double th = tanh(GELU_C * (x + GELU_A * x * x * x));
    return 0.5 * (1.0 + th) + 0.5 * x * (1.0 - th * th) * GELU_C * (1.0 + 3.0 * GELU_A * x * x);
}
static double bf16_round(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

void or_mlp_forward(const double* Pm, const double* X, int64_t B, int round_act, double* out)
{
    const double *W1 = Pm, *b1 = W1 + OR_NH * OR_NF, *W2 = b1 + OR_NH, *b2 = W2 + OR_NH * OR_NH,
                 *W3 = b2 + OR_NH, *b3 = W3 + OR_NH;
    double h1[OR_NH], h2[OR_NH];
    for (int64_t r = 0; r < B; ++r) {
        const double* x = X + r * OR_NF;
        for (int o = 0; o < OR_NH; ++o) {
            double z = b1[o];
            for (int i = 0; i < OR_NF; ++i) z += W1[o * OR_NF + i] * x[i];
            h1[o] = round_act ? bf16_round(gelu(z)) : gelu(z);
        }
        for (int o = 0; o < OR_NH; ++o) {
            double z = b2[o];
            for (int i = 0; i < OR_NH; ++i) z += W2[o * OR_NH + i] * h1[i];
            h2[o] = round_act ? bf16_round(gelu(z)) : gelu(z);
        }
        double y = b3[0];
        for (int i = 0; i < OR_NH; ++i) y += W3[i] * h2[i];
        out[r] = y;
    }
}

/* Forward of one row keeping the pre-activations z and activations h. */
static double mlp_row(const double* Pm, const double* x, double* z1, double* h1, double* z2, double* h2)
{
    const double *W1 = Pm, *b1 = W1 + OR_NH * OR_NF, *W2 = b1 + OR_NH, *b2 = W2 + OR_NH * OR_NH,
                 *W3 = b2 + OR_NH, *b3 = W3 + OR_NH;
    for (int o = 0; o < OR_NH; ++o) {
        double z = b1[o];
        for (int i = 0; i < OR_NF; ++i) z += W1[o * OR_NF + i] * x[i];
        z1[o] = z;
        h1[o] = gelu(z);
    }
    for (int o = 0; o < OR_NH; ++o) {
        double z = b2[o];
        for (int i = 0; i < OR_NH; ++i) z += W2[o * OR_NH + i] * h1[i];
        z2[o] = z;
        h2[o] = gelu(z);
    }
    double y = b3[0];
    for (int i = 0; i < OR_NH; ++i) y += W3[i] * h2[i];
    return y;
}

/* Adds dy * dy/dparams of one row to G (back-propagation through the three
 * layers by the chain rule). */
static void mlp_row_backward(const double* Pm, const double* x, double dy, double* G)
{
    const double *W2 = Pm + OR_NH * OR_NF + OR_NH, *W3 = W2 + OR_NH * OR_NH + OR_NH;
    double *gW1 = G, *gb1 = gW1 + OR_NH * OR_NF, *gW2 = gb1 + OR_NH, *gb2 = gW2 + OR_NH * OR_NH,
           *gW3 = gb2 + OR_NH, *gb3 = gW3 + OR_NH;
    double z1[OR_NH], h1[OR_NH], z2[OR_NH], h2[OR_NH], d2[OR_NH], d1[OR_NH];
    mlp_row(Pm, x, z1, h1, z2, h2);
    gb3[0] += dy;
    for (int i = 0; i < OR_NH; ++i) {
        gW3[i] += dy * h2[i];
        d2[i] = dy * W3[i] * gelu_d(z2[i]);
    }
    for (int o = 0; o < OR_NH; ++o) {
        gb2[o] += d2[o];
        for (int i = 0; i < OR_NH; ++i) gW2[o * OR_NH + i] += d2[o] * h1[i];
    }
    for (int i = 0; i < OR_NH; ++i) {
        double s = 0;
        for (int o = 0; o < OR_NH; ++o) s += W2[o * OR_NH + i] * d2[o];
        d1[i] = s * gelu_d(z1[i]);
    }
    for (int o = 0; o < OR_NH; ++o) {
        gb1[o] += d1[o];
        for (int i = 0; i < OR_NF; ++i) gW1[o * OR_NF + i] += d1[o] * x[i];
    }
}

/* Training losses and their gradients dL/dparams (G, OR_NPARAM doubles).
 * group == NULL: L = (1/B) sum_r (y_r - t_r)^2.
 * group != NULL: rows come in contiguous groups (the candidates of one step;
 * group[r] = index within the group << 16 | group size) and
 * L = (1/B) sum_r ((y_r - t_r) - mean over r's group of (y - t))^2, the squared
 * error after removing each step's common offset, which the proposal of
 * Eq. 3 cannot see (it is proportional within a step).  Its gradient is
 * dL/dy_r = (2/B) (e_r - mean_group e) because the centred residuals of a
 * group sum to zero. */
double or_mlp_grad_ex(const double* Pm, const double* X, const double* Tg, const uint32_t* group, int64_t B,
                      double* G)
{
    memset(G, 0, sizeof(double) * OR_NPARAM);
    double z1[OR_NH], h1[OR_NH], z2[OR_NH], h2[OR_NH];
    double* e = (double*)xcalloc((size_t)(B > 0 ? B : 1), sizeof(double));
    for (int64_t r = 0; r < B; ++r) e[r] = mlp_row(Pm, X + r * OR_NF, z1, h1, z2, h2) - Tg[r];
    double loss = 0;
    for (int64_t r = 0; r < B; ++r) {
        double c = e[r];
        if (group) {
            const int64_t q = group[r] >> 16, size = group[r] & 0xFFFFu, s0 = r - q;
            double mean = 0;
            for (int64_t k = 0; k < size; ++k) mean += e[s0 + k];
            c -= mean / (double)size;
        }
        loss += c * c / (double)B;
        mlp_row_backward(Pm, X + r * OR_NF, 2.0 * c / (double)B, G);
    }
    free(e);
    return loss;
}

double or_mlp_grad(const double* Pm, const double* X, const double* Tg, int64_t B, double* G)
{
    return or_mlp_grad_ex(Pm, X, Tg, NULL, B, G);
}

static void run_trajectory(or_traj* T, uint64_t seed, uint64_t traj, uint32_t matrix,
                           int32_t* chosen /* [n][2] or NULL */, int32_t* degv /* [n] or NULL */,
                           or_forced* F, or_learn* Ln, or_traj_result* res)
{
    const or_prep* P = T->P;
    const int n = P->n;
    const int fp32 = P->fp32;
    const or_schedule* s = &P->s;
    memset(res, 0, sizeof(*res));
    res->dead_step = -1;
    if (chosen) for (int t = 0; t < n; ++t) chosen[2 * t] = chosen[2 * t + 1] = -1;
    if (degv) for (int t = 0; t < n; ++t) degv[t] = -1;
    if (!P->ok) { res->log_x = -INFINITY; res->dead_step = 0; res->dead_reason = 2; return; }

    memset(T->act, 1, 2 * (size_t)n);
    memcpy(T->mask, P->mask0, (size_t)P->m);
    memcpy(T->r, P->r0, (size_t)n * 8);
    memcpy(T->c, P->c0, (size_t)n * 8);
    recompute_degrees(T);
    double log_x = 0.0;
    double track = 1.0;
    const double theta = rnd(fp32, s->theta);

    for (int t = 0; t < n; ++t) {
        if (P->max_steps > 0 && t >= P->max_steps) break;  /* prefix replay for large n */
        /* vertex selection R_V */
        int v = -1;
        if (s->vertex_rule == VR_ROW_ORDER) {
            for (int i = 0; i < n; ++i) if (T->act[i]) { v = i; break; }
        } else {
            for (int x = 0; x < 2 * n; ++x) {
                if (!T->act[x]) continue;
                if (v < 0 || T->deg[x] < T->deg[v]) v = x;   /* strict <: lowest id wins ties */
            }
        }
        const int v_is_row = v < n;
        if (degv) degv[t] = T->deg[v];
        if (T->deg[v] == 0) { res->log_x = -INFINITY; res->dead_step = t; res->dead_reason = 1; return; }

        /* candidate neighbours in adjacency order and their scores (Eq. 3) */
        int nc = 0;
        if (v_is_row) {
            for (int64_t e = P->rp[v]; e < P->rp[v + 1]; ++e)
                if (edge_live(T, e, v, P->ci[e])) { T->cand_e[nc] = e; T->cand_p[nc] = P->ci[e]; ++nc; }
        } else {
            int j = v - n;
            for (int64_t k = P->cp[j]; k < P->cp[j + 1]; ++k)
                if (edge_live(T, P->ce[k], P->ri[k], j)) { T->cand_e[nc] = P->ce[k]; T->cand_p[nc] = P->ri[k]; ++nc; }
        }
        /* nc == deg[v] by construction of deg[] */
        double smax = 0.0;
        double* sc = T->newr;  /* scratch of size n */
        if (Ln && Ln->rec_feat && !Ln->rec_full) {
            /* (features, SK target) pairs of this step.  A pair is kept only
             * if every value is finite (an SK scale can run to 0 or infinity
             * on a residual without total support); a step contributes its
             * kept pairs together, and only if there are at least two of
             * them (one candidate says nothing about the proposal's shape),
             * so the pairs of a step form one contiguous group. */
            double sum_v = 0;
            for (int q = 0; q < nc; ++q) sum_v += T->deg[v_is_row ? n + T->cand_p[q] : T->cand_p[q]];
            float* fbuf = T->recbuf;
            float* tbuf = fbuf + (size_t)nc * OR_NF;
            int* qbuf = (int*)(tbuf + nc);
            int kept = 0;
            for (int q = 0; q < nc; ++q) {
                const int l = v_is_row ? n + T->cand_p[q] : T->cand_p[q];
                float* f = fbuf + (size_t)kept * OR_NF;
                edge_features(T, t, v, l, T->cand_e[q], sum_v, f);
                const double sv_ = v_is_row ? T->r[v] : T->c[v - n];
                const double sl_ = v_is_row ? T->c[T->cand_p[q]] : T->r[T->cand_p[q]];
                const float tgt = (float)log(sv_ * sl_);
                int finite = isfinite(tgt);
                for (int z = 0; z < OR_NF; ++z) finite = finite && isfinite(f[z]);
                if (!finite) continue;
                tbuf[kept] = tgt;
                qbuf[kept] = q;
                ++kept;
            }
            if (kept >= 2 && Ln->rec_n + kept > Ln->rec_cap) Ln->rec_full = 1;
            if (kept >= 2 && !Ln->rec_full) {
                for (int i = 0; i < kept; ++i) {
                    const int64_t pos = Ln->rec_n + i;
                    memcpy(Ln->rec_feat + pos * OR_NF, fbuf + (size_t)i * OR_NF, sizeof(float) * OR_NF);
                    Ln->rec_target[pos] = tbuf[i];
                    Ln->rec_key[pos] = (traj << 28) | ((uint64_t)t << 14) | (uint64_t)qbuf[i];
                    if (Ln->rec_group) Ln->rec_group[pos] = ((uint32_t)i << 16) | (uint32_t)kept;
                }
                Ln->rec_n += kept;
            }
        }
        if (Ln && Ln->ext_logits && nc > Ln->lstride) {  /* more candidates than logits supplied */
            res->log_x = -INFINITY; res->dead_step = t; res->dead_reason = 4; return;
        }
        float* lg_model = NULL;
        if (Ln && Ln->model) {  /* logits of the network: BF16-rounded inputs and activations */
            double sum_v = 0;
            for (int q = 0; q < nc; ++q) sum_v += T->deg[v_is_row ? n + T->cand_p[q] : T->cand_p[q]];
            lg_model = (float*)T->newc;  /* scratch of n doubles holds n floats */
            for (int q = 0; q < nc; ++q) {
                const int l = v_is_row ? n + T->cand_p[q] : T->cand_p[q];
                float f[OR_NF];
                double x[OR_NF], y;
                edge_features(T, t, v, l, T->cand_e[q], sum_v, f);
                for (int z = 0; z < OR_NF; ++z) x[z] = bf16_round((double)f[z]);
                or_mlp_forward(Ln->model, x, 1, 1, &y);
                lg_model[q] = (float)y;
            }
        }
        if (lg_model && Ln->model_logits_out)
            for (int q = 0; q < nc && q < Ln->lstride; ++q)
                Ln->model_logits_out[(int64_t)t * Ln->lstride + q] = lg_model[q];
        for (int q = 0; q < nc; ++q) {
            double sv;
            if (Ln && Ln->ext_logits) {  /* supplied logits take precedence */
                const float ex = or_exp_score(Ln->ext_logits[(int64_t)t * Ln->lstride + q]);
                sv = P->val ? (double)((float)entry(P, T->cand_e[q]) * ex) : (double)ex;
            } else if (lg_model) {
                const float ex = or_exp_score(lg_model[q]);
                sv = P->val ? (double)((float)entry(P, T->cand_e[q]) * ex) : (double)ex;
            } else {
                double scale = v_is_row ? T->c[T->cand_p[q]] : T->r[T->cand_p[q]];
                sv = rnd(fp32, entry(P, T->cand_e[q]) * scale);
            }
            if (!(sv >= 0)) sv = 0;           /* NaN guard */
            sc[q] = sv;
            if (sv > smax) smax = sv;
        }
        const int k = 40 - bitlen32((uint32_t)nc);
        uint64_t W = 0;
        for (int q = 0; q < nc; ++q) {
            double ratio = rnd(fp32, sc[q] / smax);
            double x = ldexp(ratio, k);       /* exact power-of-two scaling */
            T->w[q] = (x >= 1.0) ? (uint64_t)x : 1u;
            W += T->w[q];
        }
        int pick = -1;
        if (F && F->forced) {
            if (t >= F->n_forced) {
                F->need_choice = 1;
                F->n_cand = nc;
                for (int q = 0; q < nc; ++q) F->w_out[q] = T->w[q];
                F->W_out = W;
                if (F->logx_prefix) *F->logx_prefix = log_x;
                res->log_x = log_x;
                return;
            }
            pick = F->forced[t];
        } else {
            int64_t rv = or_uniform_below(W, seed, traj, matrix, (uint32_t)t);
            if (rv < 0) { res->log_x = -INFINITY; res->dead_step = t; res->dead_reason = 3; return; }
            uint64_t acc = 0;
            for (int q = 0; q < nc; ++q) {
                acc += T->w[q];
                if (acc > (uint64_t)rv) { pick = q; break; }
            }
        }
        const int64_t ech = T->cand_e[pick];
        const int u = v_is_row ? (n + T->cand_p[pick]) : T->cand_p[pick];
        const int R = v_is_row ? v : u;          /* matched row */
        const int C = v_is_row ? u - n : v - n;  /* matched column */
        if (chosen) { chosen[2 * t] = v; chosen[2 * t + 1] = u; }

        /* correction X <- X * B_vu / q(u|v), q = w_u / W */
        double f = log((double)W) - log((double)T->w[pick]);
        if (P->val) f += log(entry(P, ech));
        log_x += f;
        const double z = rnd(fp32, T->r[R] * T->c[C]);

        /* N_t(R)\{C} and N_t(C)\{R}, then eliminate R and C */
        int cntC = 0, cntR = 0;
        for (int64_t e = P->rp[R]; e < P->rp[R + 1]; ++e) {
            int j = P->ci[e];
            if (j != C && edge_live(T, e, R, j)) T->nbrC[cntC++] = j;
        }
        for (int64_t kk = P->cp[C]; kk < P->cp[C + 1]; ++kk) {
            int i = P->ri[kk];
            if (i != R && edge_live(T, P->ce[kk], i, C)) T->nbrR[cntR++] = i;
        }
        T->act[R] = 0;
        T->act[n + C] = 0;
        for (int q = 0; q < cntC; ++q) T->deg[n + T->nbrC[q]]--;
        for (int q = 0; q < cntR; ++q) T->deg[T->nbrR[q]]--;
        track = rnd(fp32, track * z);

        if (t + 1 < n) {
            int run_dm = (s->dm == DM_ALL) || (s->dm == DM_THRS && z < theta) ||
                         (s->dm == DM_TRCK && track < theta);
            if (run_dm) {
                res->n_dm++;
                if (!dm_filter(T)) {
                    res->log_x = -INFINITY; res->dead_step = t; res->dead_reason = 2; return;
                }
                track = 1.0;
            }
            if (s->sk == SK_FIXED) {
                for (int q = 0; q < s->K; ++q) sk_sweep(T);
                res->n_full_sk += s->K;
            } else if (s->sk == SK_ADAPTIVE) {
                double a = rnd(fp32, 1.0 - z);
                double b = rnd(fp32, a * (double)s->K);
                int nit = (b > 0) ? (int)ceil(b) : 0;
                for (int q = 0; q < nit; ++q) sk_sweep(T);
                res->n_full_sk += nit;
            } else if (s->sk == SK_LOCAL) {
                local_repair(T, T->nbrR, cntR, T->nbrC, cntC, s->local_cap,
                             s->local_cap > 0 ? or_draw_u64(seed, traj, matrix, (uint32_t)t, OR_LOCAL_DRAW) : 0);
                res->n_local_sk++;
            }
        }
    }
    res->log_x = log_x;
    if (F) F->need_choice = 0;
}

/* Forced-choice replay for exhaustive enumeration (single trajectory). */
int or_forced_run(const or_prep* P, const int32_t* forced, int32_t n_forced, uint64_t* w_out,
                  uint64_t* W_out, int32_t* n_cand, double* log_x, int32_t* dead_step,
                  int32_t* chosen /* [n][2] or NULL */, int32_t* counts /* [3] or NULL */,
                  const float* ext_logits /* [n][lstride] or NULL */, int32_t lstride)
{
    or_traj* T = traj_alloc(P);
    or_forced F;
    memset(&F, 0, sizeof(F));
    F.forced = forced;
    F.n_forced = n_forced;
    F.w_out = w_out;
    or_traj_result res;
    or_learn L;
    memset(&L, 0, sizeof(L));
    L.ext_logits = ext_logits;
    L.lstride = lstride;
    run_trajectory(T, 0, 0, 0, chosen, NULL, &F, ext_logits ? &L : NULL, &res);
    traj_free(T);
    *W_out = F.W_out;
    *n_cand = F.n_cand;
    *log_x = res.log_x;
    *dead_step = res.dead_step;
    if (counts) { counts[0] = res.n_dm; counts[1] = res.n_full_sk; counts[2] = res.n_local_sk; }
    return F.need_choice;
}

/* ------------------------------------------------------------------------- */
/* Driver: trajectories first_traj .. first_traj + count - 1 over nthreads     */
/* ------------------------------------------------------------------------- */

typedef struct {
    const or_prep* P;
    uint64_t seed, first;
    uint32_t matrix;
    int64_t lo, hi;
    double* log_x;
    int32_t* dead_step;
    int32_t* chosen;  /* [count][n][2] or NULL */
    int32_t* degv;    /* [count][n] or NULL */
    const float* ext_logits;  /* [count][n][lstride] or NULL */
    int32_t lstride;
    const double* model;      /* network parameters or NULL */
    float* model_logits;      /* [count][n][lstride] or NULL: the network's logits along the path */
    int64_t counts[3];
} or_job;

static void* job_main(void* arg)
{
    or_job* J = (or_job*)arg;
    const int n = J->P->n;
    or_traj* T = traj_alloc(J->P);
    for (int64_t q = J->lo; q < J->hi; ++q) {
        or_traj_result res;
        or_learn L;
        memset(&L, 0, sizeof(L));
        L.lstride = J->lstride;
        if (J->ext_logits) L.ext_logits = J->ext_logits + q * (int64_t)n * J->lstride;
        L.model = J->model;
        if (J->model_logits) L.model_logits_out = J->model_logits + q * (int64_t)n * J->lstride;
        run_trajectory(T, J->seed, J->first + (uint64_t)q, J->matrix,
                       J->chosen ? J->chosen + q * 2 * n : NULL,
                       J->degv ? J->degv + q * n : NULL, NULL,
                       (J->ext_logits || J->model) ? &L : NULL, &res);
        J->log_x[q] = res.log_x;
        if (J->dead_step) J->dead_step[q] = res.dead_step;
        J->counts[0] += res.n_dm;
        J->counts[1] += res.n_full_sk;
        J->counts[2] += res.n_local_sk;
    }
    traj_free(T);
    return NULL;
}

void or_run_ext(const or_prep* P, uint64_t seed, uint32_t matrix, uint64_t first_traj, int64_t count,
                int nthreads, double* log_x, int32_t* dead_step, int32_t* chosen, int32_t* degv,
                int64_t* op_counts, const float* ext_logits, int32_t lstride);

void or_run(const or_prep* P, uint64_t seed, uint32_t matrix, uint64_t first_traj, int64_t count,
            int nthreads, double* log_x, int32_t* dead_step, int32_t* chosen, int32_t* degv,
            int64_t* op_counts /* [3]: DM calls, full SK sweeps, local repairs */)
{
    or_run_ext(P, seed, matrix, first_traj, count, nthreads, log_x, dead_step, chosen, degv, op_counts, NULL, 0);
}

/* Trajectories lo..hi of one call spread over nthreads host threads: plain,
 * with supplied logits (ext_logits), with this side's network (model) or
 * both (the network's logits then go to model_logits). */
static void run_jobs(const or_prep* P, uint64_t seed, uint32_t matrix, uint64_t first_traj, int64_t count,
                     int nthreads, double* log_x, int32_t* dead_step, int32_t* chosen, int32_t* degv,
                     int64_t* op_counts, const float* ext_logits, int32_t lstride, const double* model,
                     float* model_logits)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > count) nthreads = count > 0 ? (int)count : 1;
    or_job* jobs = (or_job*)xcalloc(nthreads, sizeof(or_job));
    pthread_t* th = (pthread_t*)xcalloc(nthreads, sizeof(pthread_t));
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].P = P; jobs[t].seed = seed; jobs[t].first = first_traj; jobs[t].matrix = matrix;
        jobs[t].lo = count * t / nthreads; jobs[t].hi = count * (t + 1) / nthreads;
        jobs[t].log_x = log_x; jobs[t].dead_step = dead_step; jobs[t].chosen = chosen;
        jobs[t].degv = degv;
        jobs[t].ext_logits = ext_logits;
        jobs[t].lstride = lstride;
        jobs[t].model = model;
        jobs[t].model_logits = model_logits;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, job_main, &jobs[t]);
    job_main(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    if (op_counts) {
        op_counts[0] = op_counts[1] = op_counts[2] = 0;
        for (int t = 0; t < nthreads; ++t)
            for (int q = 0; q < 3; ++q) op_counts[q] += jobs[t].counts[q];
    }
    free(jobs);
    free(th);
}

/* or_run with the learned proposal's logits supplied per trajectory and step
 * (ext_logits[count][n][lstride], candidate q of step t in adjacency order). */
void or_run_ext(const or_prep* P, uint64_t seed, uint32_t matrix, uint64_t first_traj, int64_t count,
                int nthreads, double* log_x, int32_t* dead_step, int32_t* chosen, int32_t* degv,
                int64_t* op_counts, const float* ext_logits, int32_t lstride)
{
    run_jobs(P, seed, matrix, first_traj, count, nthreads, log_x, dead_step, chosen, degv, op_counts, ext_logits,
             lstride, NULL, NULL);
}

/* Paths that follow supplied logits (ext_logits, as or_run_ext) while the
 * network with parameters `model` is evaluated at every step on this side's
 * own features: its logits go to model_logits[count][n][lstride] (candidate
 * q < lstride of step t in adjacency order), so a device network can be
 * compared with this one on exactly the states the device visited. */
void or_run_ext_model(const or_prep* P, uint64_t seed, uint32_t matrix, uint64_t first_traj, int64_t count,
                      int nthreads, double* log_x, int32_t* dead_step, int32_t* chosen, int32_t* degv,
                      const float* ext_logits, int32_t lstride, const double* model, float* model_logits)
{
    run_jobs(P, seed, matrix, first_traj, count, nthreads, log_x, dead_step, chosen, degv, NULL, ext_logits,
             lstride, model, model_logits);
}

/* Trajectories of the learned proposal computed here: features, the FP64
 * network (inputs and hidden activations rounded to bfloat16 as the tensor
 * cores see them) and the binary32 score exponent.  Statistically the same
 * estimator as the device's; not bit-identical (accumulation order). */
void or_run_model(const or_prep* P, uint64_t seed, uint32_t matrix, uint64_t first_traj, int64_t count,
                  int nthreads, double* log_x, int32_t* dead_step, int64_t* op_counts, const double* model)
{
    run_jobs(P, seed, matrix, first_traj, count, nthreads, log_x, dead_step, NULL, NULL, op_counts, NULL, 0, model,
             NULL);
}

/* (features, target) pairs of trajectories first..first+count-1 of the
 * prepared schedule (one thread, trajectory order), the kept pairs of a step
 * contiguous with group[] = index within the step << 16 | the step's count
 * (group may be NULL).  Recording stops at the first step whose pairs do not
 * all fit in cap.  Returns the pair count. */
int64_t or_record(const or_prep* P, uint64_t seed, uint32_t matrix, uint64_t first, int64_t count,
                  int64_t cap, float* feat, float* target, uint64_t* key, uint32_t* group)
{
    or_traj* T = traj_alloc(P);
    or_learn L;
    memset(&L, 0, sizeof(L));
    L.rec_feat = feat;
    L.rec_target = target;
    L.rec_key = key;
    L.rec_group = group;
    L.rec_cap = cap;
    for (int64_t q = 0; q < count && !L.rec_full; ++q) {
        or_traj_result res;
        run_trajectory(T, seed, first + (uint64_t)q, matrix, NULL, NULL, NULL, &L, &res);
    }
    traj_free(T);
    return L.rec_n;
}

/* DM of a whole matrix with an explicit edge mask (for pins): returns 0 if no
 * perfect matching, else writes the supported-edge mask. */
int or_dm_mask(const or_prep* P, uint8_t* mask_out)
{
    or_traj* T = traj_alloc(P);
    memset(T->act, 1, 2 * (size_t)P->n);
    memset(T->mask, 1, (size_t)P->m);
    recompute_degrees(T);
    int ok = dm_filter(T);
    memcpy(mask_out, T->mask, (size_t)P->m);
    traj_free(T);
    return ok;
}

/* K full SK iterations from r = c = 1 on the whole matrix (for pins). */
void or_sk_full(const or_prep* P, int iters, double* r, double* c)
{
    or_traj* T = traj_alloc(P);
    memset(T->act, 1, 2 * (size_t)P->n);
    memset(T->mask, 1, (size_t)P->m);
    recompute_degrees(T);
    for (int v = 0; v < P->n; ++v) { T->r[v] = 1.0; T->c[v] = 1.0; }
    for (int k = 0; k < iters; ++k) sk_sweep(T);
    memcpy(r, T->r, (size_t)P->n * 8);
    memcpy(c, T->c, (size_t)P->n * 8);
    traj_free(T);
}

/* ------------------------------------------------------------------------- */
/* Statistics (Sec. 2, Sec. 3.2, Sec. 4 "Metrics"), all zero contributions     */
/* included.  X_k = exp(log_x[k]); values are shifted by the largest log so   */
/* nothing overflows: y_k = exp(log_x[k] - c).                                 */
/* ------------------------------------------------------------------------- */

typedef struct {
    double log_estimate;  /* ln mean(X); -inf if every X is 0 */
    double p_match;       /* #{X > 0} / M */
    double rel_spread;    /* s_X / |mean X|, s_X with M - 1 */
    double rse;           /* rel_spread / sqrt(M) */
    double ess;           /* (sum X)^2 / sum X^2 */
    double log_sum_x;     /* ln sum X */
    double log_sum_x2;    /* ln sum X^2 */
    int64_t n_alive;
} or_stats;

void or_statistics(const double* log_x, int64_t M, or_stats* out)
{
    memset(out, 0, sizeof(*out));
    double c = -INFINITY;
    int64_t alive = 0;
    for (int64_t k = 0; k < M; ++k) {
        if (log_x[k] > -INFINITY) { ++alive; if (log_x[k] > c) c = log_x[k]; }
    }
    out->n_alive = alive;
    out->p_match = M ? (double)alive / (double)M : 0.0;
    if (alive == 0) {
        out->log_estimate = out->log_sum_x = out->log_sum_x2 = -INFINITY;
        out->rel_spread = out->rse = NAN;
        out->ess = 0;
        return;
    }
    double sy = 0, sy2 = 0;
    for (int64_t k = 0; k < M; ++k) {
        double y = (log_x[k] > -INFINITY) ? exp(log_x[k] - c) : 0.0;
        sy += y;
        sy2 += y * y;
    }
    double mean = sy / (double)M;
    double ss = 0;
    for (int64_t k = 0; k < M; ++k) {
        double y = (log_x[k] > -INFINITY) ? exp(log_x[k] - c) : 0.0;
        ss += (y - mean) * (y - mean);
    }
    double sd = (M > 1) ? sqrt(ss / (double)(M - 1)) : NAN;
    out->log_estimate = c + log(mean);
    out->log_sum_x = c + log(sy);
    out->log_sum_x2 = 2 * c + log(sy2);
    out->rel_spread = sd / mean;
    out->rse = out->rel_spread / sqrt((double)M);
    out->ess = sy * sy / sy2;
}
