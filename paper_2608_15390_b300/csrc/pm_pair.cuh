// pm_pair.cuh -- two trajectories per warp (included by pm_traj.cu).
//
// The plain and learned schedules (no inner SK, DM or Local repair, state in
// shared memory) spend most of a step on warp-wide scans, ballots and
// reductions over the picked vertex's few candidates (degree 4-8 at these
// workloads), so most lanes of a one-trajectory warp idle while the step's
// dependency chain sets the pace.  Here each half-warp (a 16-lane segment)
// carries its own trajectory: both segments run the same instruction stream,
// every loop runs the larger of their trip counts with per-segment
// predicates, and every collective is segmented (xor / up shuffles inside a
// half, ballots masked to the half).  Per trajectory the arithmetic is that
// of run_group -- the same picks, integer weights, draws, corrections and
// network logits -- so every trajectory's ln X is bit-identical to the
// one-trajectory-per-warp kernel's.  The network evaluates both segments'
// candidate tiles in one interleaved pass that shares the weight fragments.
// When both candidate lists fit one 16-lane chunk (the common case), each
// candidate is read, scored and weighted once for the whole step.  The file
// is included inside pm_traj.cu's anonymous namespace, after the step
// helpers it shares with run_group; the scaled and uniform proposals also
// run it in the 24-warp pair-only kernel.

struct Seg {
    int h;         // segment (0: lanes 0-15, 1: lanes 16-31)
    int sl;        // lane within the segment
    int base;      // first lane of the segment
};

__device__ __forceinline__ unsigned seg_ballot(const Seg& S, bool p)
{
    return (__ballot_sync(kFull, p) >> S.base) & 0xFFFFu;
}
template <typename T>
__device__ __forceinline__ T seg_shfl(const Seg& S, T v, int src)
{
    return __shfl_sync(kFull, v, S.base + src);
}
// the larger of the two segments' values of x (every lane gets it)
__device__ __forceinline__ int both_max(int x)
{
    const int o = __shfl_xor_sync(kFull, x, 16);
    return x > o ? x : o;
}
__device__ __forceinline__ uint32_t seg_min_u32(uint32_t v)
{
#pragma unroll
    for (int o = 8; o; o >>= 1) {
        const uint32_t t = __shfl_xor_sync(kFull, v, o);
        v = t < v ? t : v;
    }
    return v;
}
__device__ __forceinline__ unsigned long long seg_min_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 8; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(kFull, v, o);
        v = t < v ? t : v;
    }
    return v;
}
__device__ __forceinline__ int seg_sum_int(int v)
{
#pragma unroll
    for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ int seg_max_int(int v)
{
#pragma unroll
    for (int o = 8; o; o >>= 1) {
        const int t = __shfl_xor_sync(kFull, v, o);
        v = t > v ? t : v;
    }
    return v;
}
// lists at most this long are summed by their own lane (nbr_degree_sum_seg)
constexpr int kSerialList = 24;
__device__ __forceinline__ uint64_t seg_sum_u64(uint64_t v)
{
#pragma unroll
    for (int o = 8; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ unsigned seg_or(unsigned v)
{
#pragma unroll
    for (int o = 8; o; o >>= 1) v |= __shfl_xor_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ uint64_t seg_incl_scan_u64(uint64_t v, int sl)
{
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const uint64_t t = __shfl_up_sync(kFull, v, o, 16);
        if (sl >= o) v += t;
    }
    return v;
}
__device__ __forceinline__ int seg_incl_scan_int(int v, int sl)
{
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const int t = __shfl_up_sync(kFull, v, o, 16);
        if (sl >= o) v += t;
    }
    return v;
}
// maximum of non-negative values inside a segment (IEEE bit patterns order as integers)
__device__ __forceinline__ float seg_max_nonneg(float v)
{
    uint32_t b = __float_as_uint(v);
#pragma unroll
    for (int o = 8; o; o >>= 1) {
        const uint32_t t = __shfl_xor_sync(kFull, b, o);
        b = t > b ? t : b;
    }
    return __uint_as_float(b);
}
__device__ __forceinline__ double seg_max_nonneg(double v)
{
    long long b = __double_as_longlong(v);
#pragma unroll
    for (int o = 8; o; o >>= 1) {
        const long long t = __shfl_xor_sync(kFull, b, o);
        b = t > b ? t : b;
    }
    return __longlong_as_double(b);
}

// the active vertex of least (live degree, unified id) of the segment's tree
// (md_pick with two top-level entries per lane); `use` false: a safe 0
__device__ __forceinline__ int md_pick_seg(const uint16_t* deg, const uint32_t* tree, const TreeGeom& T, const Seg& S,
                                           bool use)
{
    uint32_t key = 0xFFFFFFFFu;
    int top_off = 0, top_size = T.n2;
#pragma unroll
    for (int l = 1; l <= kMaxTreeLevels; ++l)
        if (l == T.nlev) { top_off = T.off[l]; top_size = T.size[l]; }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int x = S.sl + 16 * q;
        uint32_t k2 = 0xFFFFFFFFu;
        if (T.nlev == 0) { if (x < T.n2) k2 = leaf_key(deg, x, T); }
        else if (x < top_size) k2 = tree[top_off + x];
        key = k2 < key ? k2 : key;
    }
    key = seg_min_u32(key);
    const bool sat = (key >> T.idb) >= T.dcap;
    int v = (int)(key & ((1u << T.idb) - 1u));
    if (__any_sync(kFull, sat && use)) {  // a saturated degree field: exact scan (both segments, uniform loop)
        unsigned long long best = ~0ull;
        for (int x = S.sl; x < T.n2; x += 16) {
            const uint32_t d = deg[x];
            if (d == kInact) continue;
            const unsigned long long k64 = ((unsigned long long)d << 32) | (unsigned)x;
            best = k64 < best ? k64 : best;
        }
        best = seg_min_u64(best);
        if (sat) v = (int)(best & 0xFFFFFFFFu);
    }
    return use ? v : 0;
}

// recompute the tree entries above leaves x and y of the segment's tree
// (tree_fix2 with two children per lane); `use` false: loads only, no stores
__device__ void tree_fix2_seg(const uint16_t* deg, uint32_t* tree, const TreeGeom& T, int x, int y, const Seg& S,
                              bool use)
{
#pragma unroll
    for (int l = 1; l <= kMaxTreeLevels; ++l) {
        if (l > T.nlev) break;
        const int gx = x >> (5 * l), gy = y >> (5 * l);
        const bool two = gy != gx;
        uint32_t kx = 0xFFFFFFFFu, ky = 0xFFFFFFFFu;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int cx = gx * 32 + S.sl + 16 * q, cy = gy * 32 + S.sl + 16 * q;
            uint32_t a = 0xFFFFFFFFu, b = 0xFFFFFFFFu;
            if (cx < T.size[l - 1]) a = (l == 1) ? leaf_key(deg, cx, T) : tree[T.off[l - 1] + cx];
            if (two && cy < T.size[l - 1]) b = (l == 1) ? leaf_key(deg, cy, T) : tree[T.off[l - 1] + cy];
            kx = a < kx ? a : kx;
            ky = b < ky ? b : ky;
        }
        kx = seg_min_u32(kx);
        ky = seg_min_u32(ky);
        if (use && S.sl == 0) {
            tree[T.off[l] + gx] = kx;
            if (two) tree[T.off[l] + gy] = ky;
        }
        __syncwarp();
    }
}

// neighbour_degree_sum_flat for a segment: the degree sums over the live
// neighbours of each live candidate of the chunk (lane sl holds candidate
// sl).  Short lists are summed by their own lane; otherwise one pass over the
// concatenated lists of both segments' candidates, lane f taking entry f;
// acc: 16 ints of the segment's shared scratch.  Integer sums: identical to
// neighbour_degree_sum.
template <typename Idx>
__device__ __forceinline__ int nbr_degree_sum_seg(const MV<Idx>& V, const uint16_t* deg, const uint8_t* mask, bool vrow,
                                                  int pp, bool live, const Seg& S, int* acc, int& entries)
{
    const int n = V.n;
    int b = 0, len = 0;
    if (live) {
        b = vrow ? V.cp[pp] : V.rp[pp];
        len = (vrow ? V.cp[pp + 1] : V.rp[pp + 1]) - b;
    }
    // short lists (every list of both segments at most kSerialList entries):
    // each lane sums its own candidate's list, no cross-lane traffic
    const int maxlen = both_max(seg_max_int(len));
    if (maxlen <= kSerialList) {
        entries = seg_sum_int(len);
        int mine = 0;
        for (int q = 0; q < len; ++q) {
            const int pos = b + q;
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
            if (ok) mine += (int)d;
        }
        return mine;
    }
    const int incl = seg_incl_scan_int(len, S.sl);
    const int excl = incl - len;
    const int total = seg_shfl(S, incl, 15);
    entries = total;
    acc[S.sl] = 0;
    __syncwarp();
    const bool has = live && len > 0;
    const unsigned lm = seg_ballot(S, has);
    const int TOT = both_max(total);
    for (int base = 0; base < TOT; base += 16) {
        const int f = base + S.sl;
        const unsigned before = seg_ballot(S, has && excl < base);
        const unsigned starts = seg_or((has && excl >= base && excl < base + 16) ? 1u << (excl - base) : 0u);
        const int rank = __popc(before) + __popc(starts & (0xFFFFu >> (15 - S.sl)));
        const int owner = (f < total) ? (int)__fns(lm, 0, rank) : -1;
        const int src = owner >= 0 ? owner : 0;
        const int oe = seg_shfl(S, excl, src), ob = seg_shfl(S, b, src);
        if (owner >= 0) {
            const int pos = ob + (f - oe);
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
    const int mine = acc[S.sl];
    __syncwarp();
    return mine;
}

// mlp_infer8 on two 8-candidate tiles at once (fa: segment 0's, fb:
// segment 1's), one instruction stream with the weight fragments loaded
// once; per tile every instruction is mlp_infer8's, so the outputs are its
// bits.  Lane 4g (g < 8) gets candidate g's output of each tile.
__device__ __forceinline__ void mlp_infer8x2(const DevModel* M, const uint16_t* fa, const uint16_t* fb, int lane,
                                             float& ya, float& yb)
{
    const int g = lane >> 2, t = lane & 3;
    const uint32_t xa = ld32(fa + g * kFS + 2 * t), xb = ld32(fb + g * kFS + 2 * t);
    uint32_t ha[4][2], hb[4][2];
#pragma unroll
    for (int mt = 0; mt < 4; ++mt) {
        const int h0 = 16 * mt + g;
        float aa[4] = {M->b1[h0], M->b1[h0], M->b1[h0 + 8], M->b1[h0 + 8]};
        float ab[4] = {aa[0], aa[1], aa[2], aa[3]};
        const uint32_t a[4] = {ld32(M->w1p + h0 * kW1S + 2 * t), ld32(M->w1p + (h0 + 8) * kW1S + 2 * t), 0u, 0u};
        mma16816(aa, a, xa, 0u);
        mma16816(ab, a, xb, 0u);
        ha[mt][0] = trans8x8(pack_bf16(gelu_f(aa[0]), gelu_f(aa[1])));
        ha[mt][1] = trans8x8(pack_bf16(gelu_f(aa[2]), gelu_f(aa[3])));
        hb[mt][0] = trans8x8(pack_bf16(gelu_f(ab[0]), gelu_f(ab[1])));
        hb[mt][1] = trans8x8(pack_bf16(gelu_f(ab[2]), gelu_f(ab[3])));
    }
    float oa[4] = {t == 0 ? M->b3[0] : 0.f, 0.f, 0.f, 0.f};
    float ob[4] = {oa[0], 0.f, 0.f, 0.f};
#pragma unroll 2
    for (int mt = 0; mt < 4; ++mt) {
        const int h0 = 16 * mt + g;
        float aa[4] = {M->b2[h0], M->b2[h0], M->b2[h0 + 8], M->b2[h0 + 8]};
        float ab[4] = {aa[0], aa[1], aa[2], aa[3]};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            uint32_t a[4];
            ldsm_a(a, M->w2 + 16 * mt * kWS + 16 * kk, lane);
            mma16816(aa, a, ha[kk][0], ha[kk][1]);
            mma16816(ab, a, hb[kk][0], hb[kk][1]);
        }
        const uint32_t a3a[4] = {trans8x8(pack_bf16(gelu_f(aa[0]), gelu_f(aa[1]))), 0u,
                                 trans8x8(pack_bf16(gelu_f(aa[2]), gelu_f(aa[3]))), 0u};
        const uint32_t a3b[4] = {trans8x8(pack_bf16(gelu_f(ab[0]), gelu_f(ab[1]))), 0u,
                                 trans8x8(pack_bf16(gelu_f(ab[2]), gelu_f(ab[3]))), 0u};
        const uint32_t w0 = ld32(M->w3p + g * kWS + 16 * mt + 2 * t), w1 = ld32(M->w3p + g * kWS + 16 * mt + 2 * t + 8);
        mma16816(oa, a3a, w0, w1);
        mma16816(ob, a3b, w0, w1);
    }
    ya = oa[0];
    yb = ob[0];
}

// One warp, two trajectories: the trajectories of chunk `ch` claimed by
// segment, run to their ends.  MODE 0 (scaled or uniform proposal) or 1
// (learned); no inner SK, DM or Local repair; state in shared memory.
// sbase: the warp's two trajectory states of pl.state_bytes each; slot: the
// warp's global scratch (two long-list logit buffers of n_max floats).
template <typename Real, typename Idx, int MODE>
__device__ void run_pair(const TrajParams& P, const DevMatrix* Mp, const MV<Idx>& V, int k, const Chunk& ch,
                         const Plan& pl, uint8_t* sbase, uint8_t* slot, int* ctr_traj, const DevModel* Ms, int lane)
{
    constexpr bool model = MODE == 1;
    const int n = V.n;
    const uint32_t midx = (uint32_t)Mp->idx;
    const TreeGeom T = tree_geom(n);
    Seg S;
    S.h = lane >> 4;
    S.sl = lane & 15;
    S.base = 16 * S.h;
    uint8_t* base = sbase + (size_t)S.h * pl.state_bytes;
    uint16_t* deg = reinterpret_cast<uint16_t*>(base);
    size_t off = a16((size_t)((2 * n + 7) & ~7) * 2);
    uint32_t* tree = reinterpret_cast<uint32_t*>(base + off);
    off += a16((size_t)T.total * 4);
    uint16_t* feat = reinterpret_cast<uint16_t*>(base + off);  // [16][kFS] bf16 rows (learned)
    float* lgbuf = model ? reinterpret_cast<float*>(slot + P.slot.logit) + (size_t)S.h * P.n_max : nullptr;
    const Real* r = reinterpret_cast<const Real*>(Mp->r0);
    const Real* c = reinterpret_cast<const Real*>(Mp->c0);
    const bool uniform = Mp->unit_scale;

    bool has = false, done = false;
    int t = 0;
    uint64_t local = 0, traj = 0, gq = 0;
    Mant64 num, den;
    uint64_t alg_bytes = 0, mlp_rows = 0, t_begin = 0;
    for (;;) {
        // claim and start a trajectory for each segment without one (a matrix
        // without a perfect matching gives ln X = -inf at once)
        for (;;) {
            const bool need = !has && !done;
            if (!__any_sync(kFull, need)) break;
            int q = 0;
            if (need && S.sl == 0)
                q = (P.budget_ns && stop_starting(P, false)) ? (int)ch.count : atomicAdd(ctr_traj, 1);
            q = __shfl_sync(kFull, q, S.base);
            if (!need) {
            } else if (q >= (int)ch.count) {
                done = true;
            } else if (!Mp->ok) {
                if (S.sl == 0) P.log_x[ch.slot0 + (uint64_t)q] = -INFINITY;
            } else {
                has = true;
                t = 0;
                local = ch.first + (uint64_t)q;
                traj = P.first_traj + local;
                gq = ch.slot0 + (uint64_t)q;
                num = Mant64{};
                den = Mant64{};
                alg_bytes = (uint64_t)16 * n;
                mlp_rows = 0;
                t_begin = S.sl == 0 ? global_ns() : 0;
                const uint4* src = reinterpret_cast<const uint4*>(Mp->deg0);
                uint4* dst = reinterpret_cast<uint4*>(deg);
                const int nv = (2 * n + 7) / 8;
                for (int v = S.sl; v < nv; v += 16) dst[v] = __ldg(src + v);
                for (int v = S.sl; v < T.total; v += 16) tree[v] = __ldg(Mp->tree0 + v);
            }
            __syncwarp();
        }
        __syncwarp();
        if (!__any_sync(kFull, has)) break;

        // ---- one step of each running trajectory ----
        bool abandoned = false;
        if (P.hard_ns) {  // far past the budget: leave this trajectory out
            int over = 0;
            if (has && (t & 63) == 0 && S.sl == 0) {
                const unsigned long long t0 = *reinterpret_cast<volatile unsigned long long*>(P.t_start);
                over = t0 && global_ns() - t0 > P.hard_ns;
                if (over) atomicOr(P.status, ST_TIMEOUT);
            }
            abandoned = __shfl_sync(kFull, over, S.base) != 0;
        }
        const uint64_t u0 = draw_u64(P.seed, traj, midx, (uint32_t)t, 0);
        const bool vr_row = P.s.vertex_rule == VR_ROW;
        const int vm = vr_row ? 0 : md_pick_seg(deg, tree, T, S, has && !abandoned);
        int v = (vr_row && has && !abandoned) ? t : vm;
        PM_CLAMP(v, 2 * n);
        const int dv = (has && !abandoned) ? (int)deg[v] : 0;
        const bool alive = has && !abandoned && dv > 0;  // a step is taken
        const bool vrow = v < n;
        const int vi = vrow ? v : v - n;
        const int beg = alive ? (vrow ? V.rp : V.cp)[vi] : 0;
        const int end = alive ? (vrow ? V.rp : V.cp)[vi + 1] : 0;
        const auto adj = vrow ? V.ci : V.ri;
        const int poff = vrow ? n : 0;
        const int kq = 40 - bitlen((uint32_t)(dv > 0 ? dv : 1));
        const int len = end - beg;
        const int NCH = both_max((len + 15) >> 4);
        const bool net = model && alive && dv >= 2;  // a single live candidate needs no network
        // both lists fit one 16-lane chunk: this lane's candidate is read once, for the
        // network, the sampling and the elimination
        const bool one = NCH == 1;
        int pp1 = 0;
        bool live1 = false;
        if (one) {
            const int e = beg + S.sl;
            const bool in = alive && e < end;
            pp1 = in ? (int)adj[e] : 0;
            live1 = in && entry_live(deg, (const uint8_t*)nullptr, V, vrow, e, pp1 + poff);
        }

        // learned proposal: the network's logit of every live candidate
        float lg_reg = 0.f;
        if (model && __any_sync(kFull, net)) {
            float sum_v = 0.f, lsv = 0.f;
            {
                int sv_i = 0;
                if (one) {
                    if (net && live1) sv_i = deg[pp1 + poff];
                } else {
                    for (int cc = 0; cc < NCH; ++cc) {
                        const int e = beg + 16 * cc + S.sl;
                        if (net && e < end) {
                            const int pid = (int)adj[e] + poff;
                            if (entry_live(deg, (const uint8_t*)nullptr, V, vrow, e, pid)) sv_i += deg[pid];
                        }
                    }
                }
                sv_i = seg_sum_int(sv_i);
                sum_v = (float)sv_i;
                if (net) {
                    const float* s0 = reinterpret_cast<const float*>(vrow ? Mp->r0 : Mp->c0);
                    lsv = __logf(__ldg(s0 + vi));
                }
            }
            for (int cc = 0; cc < NCH; ++cc) {
                const int e = beg + 16 * cc + S.sl;
                const bool in = net && e < end;
                int pp;
                bool live;
                if (one) {
                    pp = in ? pp1 : 0;
                    live = net && live1;
                } else {
                    pp = in ? (int)adj[e] : 0;
                    live = in && entry_live(deg, (const uint8_t*)nullptr, V, vrow, e, pp + poff);
                }
                const unsigned lmk = seg_ballot(S, live);
                const int nl = __popc(lmk);
                const int li = __popc(lmk & ((1u << S.sl) - 1u));
                const CandLoads cl = cand_loads<Idx>(V, Mp, vrow, e, pp, live);
                int entries = 0;
                const int sum_l = nbr_degree_sum_seg<Idx>(V, deg, nullptr, vrow, pp, live, S,
                                                          reinterpret_cast<int*>(feat), entries);
                if (net && S.sl == 0) alg_bytes += (uint64_t)8 * entries + (uint64_t)16 * nl;
                uint16_t* f0 = reinterpret_cast<uint16_t*>(sbase + 0 * (size_t)pl.state_bytes + off);
                const uint16_t* f1 = reinterpret_cast<const uint16_t*>(sbase + 1 * (size_t)pl.state_bytes + off);
                // at most 4 live candidates in each half (the usual minimum-degree
                // pick): both halves share one 8-candidate tile of half 0, half 1
                // in rows 4-7 (each candidate's network output depends on its
                // own row of features only)
                const bool packed = both_max(nl) <= 4;
                if (live) {
                    float f[8];
                    cand_features<Idx>(V, deg, t, vrow, pp, sum_v, sum_l, (float)dv, lsv, cl, f);
                    uint4 lo;
                    lo.x = pack_bf16(f[0], f[1]);
                    lo.y = pack_bf16(f[2], f[3]);
                    lo.z = pack_bf16(f[4], f[5]);
                    lo.w = pack_bf16(f[6], f[7]);
                    uint16_t* row = packed ? f0 + (li + 4 * S.h) * kFS : feat + li * kFS;
                    *reinterpret_cast<uint4*>(row) = lo;
                }
                __syncwarp();
                float lg = 0.f;
                if (packed) {
                    const float y = mlp_infer8(Ms, f0, lane);
                    const float v = __shfl_sync(kFull, y, 4 * ((li & 3) + 4 * S.h));
                    if (live) lg = v;
                } else {
                    const int NT = both_max((nl + 7) >> 3);
                    for (int tile = 0; tile < NT; ++tile) {
                        float ya, yb;
                        mlp_infer8x2(Ms, f0 + 8 * tile * kFS, f1 + 8 * tile * kFS, lane, ya, yb);
                        const float va = __shfl_sync(kFull, ya, 4 * (li & 7)), vb = __shfl_sync(kFull, yb, 4 * (li & 7));
                        if (live && (li >> 3) == tile) lg = S.h == 0 ? va : vb;
                    }
                }
                __syncwarp();
                mlp_rows += nl;
                if (len > 16 && e < end && net) lgbuf[e - beg] = lg;
                if (cc == 0) lg_reg = lg;
            }
        }
        // score of a live candidate: B * c (scaled) or B * e^logit (learned)
        auto score = [&](int e, int pp, float lg) -> Real {
            if (!model) return cand_score<Real, Idx>(V, vrow, e, pp, r, c);
            const float* vals = vrow ? V.rv : V.cv;
            const float ex = exp_score(lg);
            Real sv = vals ? (Real)__fmul_rn(__ldg(vals + e), ex) : (Real)ex;
            if (!(sv >= (Real)0)) sv = 0;
            return sv;
        };
        auto logit_at = [&](int cc, int e) -> float {
            if (!net) return 0.f;
            return cc == 0 ? lg_reg : lgbuf[e - beg];
        };
        // the largest score, the total integer weight W, the draw and the
        // partner (the first live candidate whose prefix weight exceeds it)
        Real smax = 0;
        uint64_t W = 0, rr = 0, w_sel = 0;
        int sel_e = -1, sel_p = -1;
        bool rng_fail = false;
        if (one) {  // each candidate's weight is computed once
            const int e = beg + S.sl;
            uint64_t w = 0;
            if (uniform) {
                w = live1 ? (1ull << kq) : 0ull;
                W = alive ? ((uint64_t)dv << kq) : 0;
            } else {
                const Real sv = live1 ? score(e, pp1, logit_at(0, e)) : (Real)0;
                smax = seg_max_nonneg(sv);
                w = live1 ? quant_weight<Real>(sv, smax, kq) : 0ull;
            }
            const uint64_t pre = seg_incl_scan_u64(w, S.sl);
            if (!uniform) W = seg_shfl(S, pre, 15);
            if (alive) {
                rr = uniform_below(W, u0, P.seed, traj, midx, (uint32_t)t);
                rng_fail = rr == ~0ull;
            }
            __syncwarp();
            const unsigned hit = seg_ballot(S, live1 && !rng_fail && pre > rr);
            const int sl_hit = hit ? __ffs(hit) - 1 : 0;
            const int se = seg_shfl(S, e, sl_hit), sp = seg_shfl(S, pp1, sl_hit);
            const uint64_t sw = seg_shfl(S, w, sl_hit);
            if (hit) {
                sel_e = se;
                sel_p = sp;
                w_sel = sw;
            }
        } else {
            if (uniform) {
                W = alive ? ((uint64_t)dv << kq) : 0;
            } else {
                for (int cc = 0; cc < NCH; ++cc) {
                    const int e = beg + 16 * cc + S.sl;
                    Real sv = 0;
                    if (alive && e < end) {
                        const int pp = adj[e];
                        if (entry_live(deg, (const uint8_t*)nullptr, V, vrow, e, pp + poff))
                            sv = score(e, pp, logit_at(cc, e));
                    }
                    const Real cm = seg_max_nonneg(sv);
                    smax = cm > smax ? cm : smax;
                }
                for (int cc = 0; cc < NCH; ++cc) {
                    const int e = beg + 16 * cc + S.sl;
                    uint64_t w = 0;
                    if (alive && e < end) {
                        const int pp = adj[e];
                        if (entry_live(deg, (const uint8_t*)nullptr, V, vrow, e, pp + poff))
                            w = quant_weight<Real>(score(e, pp, logit_at(cc, e)), smax, kq);
                    }
                    W += seg_sum_u64(w);
                }
            }
            if (alive) {
                rr = uniform_below(W, u0, P.seed, traj, midx, (uint32_t)t);
                rng_fail = rr == ~0ull;
            }
            __syncwarp();
            uint64_t carry = 0;
            bool found = false;
            for (int cc = 0; cc < NCH; ++cc) {
                const int e = beg + 16 * cc + S.sl;
                int pp = 0;
                bool live = false;
                uint64_t w = 0;
                if (alive && !rng_fail && e < end) {
                    pp = adj[e];
                    live = entry_live(deg, (const uint8_t*)nullptr, V, vrow, e, pp + poff);
                    if (live) w = uniform ? (1ull << kq) : quant_weight<Real>(score(e, pp, logit_at(cc, e)), smax, kq);
                }
                const uint64_t pre = seg_incl_scan_u64(w, S.sl) + carry;
                const unsigned hit = seg_ballot(S, live && !found && pre > rr);
                const int sl_hit = hit ? __ffs(hit) - 1 : 0;
                const int se = seg_shfl(S, e, sl_hit), sp = seg_shfl(S, pp, sl_hit);
                const uint64_t sw = seg_shfl(S, w, sl_hit);
                if (hit && !found) {
                    sel_e = se;
                    sel_p = sp;
                    w_sel = sw;
                    found = true;
                }
                carry = seg_shfl(S, pre, 15);
            }
        }
        bool dead = has && !abandoned && (dv == 0 || rng_fail);
        if (rng_fail && S.sl == 0) atomicOr(P.status, ST_RNG_EXHAUSTED);
        bool stepping = alive && !rng_fail;
        if (stepping && (sel_p < 0 || sel_e < beg || sel_e >= end)) {  // only with corrupt degrees
            if (S.sl == 0) atomicOr(P.status, ST_INTERNAL);
            dead = true;
            stepping = false;
        }
        const int R = vrow ? vi : sel_p;  // matched row
        const int C = vrow ? sel_p : vi;  // matched column
        if (stepping && S.sl == 0) {  // X <- X * B_vu * W / w_u
            num.mul(W);
            const float* vals = vrow ? V.rv : V.cv;
            if (vals) num.mul(__ldg(vals + sel_e));
            den.mul(w_sel);
        }
        __syncwarp();
        if (stepping && S.sl == 0) {
            deg[R] = kInact;
            deg[n + C] = kInact;
        }
        __syncwarp();
        // eliminate: the live neighbours of v, then of the partner, lose a degree
        int cnt = 0;
        if (one) {  // the candidates live before the pick, less the partner
            const bool keep = stepping && live1 && pp1 != sel_p;
            if (keep) {
                const int pid = pp1 + poff;
                const uint32_t d = deg[pid] - 1u;
                deg[pid] = (uint16_t)d;
                tree_lower(tree, T, pid, d);
            }
            cnt += __popc(seg_ballot(S, keep));
        } else {
            for (int cc = 0; cc < NCH; ++cc) {
                const int e = beg + 16 * cc + S.sl;
                bool live = false;
                int pid = 0;
                if (stepping && e < end) {
                    pid = (int)adj[e] + poff;
                    live = entry_live(deg, (const uint8_t*)nullptr, V, vrow, e, pid);
                }
                if (live) {
                    const uint32_t d = deg[pid] - 1u;
                    deg[pid] = (uint16_t)d;
                    tree_lower(tree, T, pid, d);
                }
                cnt += __popc(seg_ballot(S, live));
            }
        }
        const bool urow = !vrow;
        const int ub = stepping ? (urow ? V.rp : V.cp)[sel_p] : 0;
        const int ue = stepping ? (urow ? V.rp : V.cp)[sel_p + 1] : 0;
        const auto uadj = urow ? V.ci : V.ri;
        const int uoff = urow ? n : 0;
        const int NU = both_max((ue - ub + 15) >> 4);
        for (int cc = 0; cc < NU; ++cc) {
            const int e = ub + 16 * cc + S.sl;
            bool live = false;
            int pid = 0;
            if (stepping && e < ue) {
                pid = (int)uadj[e] + uoff;
                live = entry_live(deg, (const uint8_t*)nullptr, V, urow, e, pid);
            }
            if (live) {
                const uint32_t d = deg[pid] - 1u;
                deg[pid] = (uint16_t)d;
                tree_lower(tree, T, pid, d);
            }
            cnt += __popc(seg_ballot(S, live));
        }
        if (stepping && S.sl == 0) {
            alg_bytes += (uint64_t)8 * (uint64_t)(len + (ue - ub)) + 16 + (uint64_t)32 * (uint64_t)cnt;
            if (!uniform && !model) alg_bytes += (uint64_t)sizeof(Real) * (uint64_t)len;
            if ((vrow ? V.rv : V.cv) != nullptr) alg_bytes += (uint64_t)4 * (uint64_t)len;
        }
        __syncwarp();
        if (!vr_row) tree_fix2_seg(deg, tree, T, stepping ? R : 0, stepping ? n + C : 0, S, stepping);
        if (stepping) ++t;
        // a finished trajectory: its result and counters
        const bool complete = stepping && t == n;
        if ((dead || complete || abandoned) && S.sl == 0) {
            if (!abandoned) P.log_x[gq] = dead ? -INFINITY : log_ratio(num, den);
            unsigned long long* ctr = P.counters + kCounters * k;
            atomicAdd(ctr + 3, (unsigned long long)alg_bytes);
            if (mlp_rows) atomicAdd(ctr + 4, (unsigned long long)mlp_rows);
            atomicAdd(ctr + 5, (unsigned long long)(global_ns() - t_begin));
        }
        if (dead || complete || abandoned) has = false;
        __syncwarp();
    }
}

// The warps of a pair plan: warp w runs trajectory states 2w and 2w + 1.
template <typename Real, typename Idx, int MODE>
__device__ void run_chunk_pair(const TrajParams& P, const Chunk& ch, const Plan& pl, const MV<Idx>& V,
                               uint8_t* gstate, int* ctr_traj, const DevModel* Ms)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (2 * warp + 1 >= pl.groups) return;
    uint8_t* sbase = gstate + (size_t)(2 * warp) * pl.state_bytes;
    uint8_t* slot = P.slots + ((size_t)blockIdx.x * P.cta_warps + warp) * P.slot.bytes;
    run_pair<Real, Idx, MODE>(P, P.mats + ch.k, V, ch.k, ch, pl, sbase, slot, ctr_traj, Ms, lane);
}

