// pm_api.cu -- host implementation of the C ABI declared in include/pm.h:
// argument checks, the context's device arena, launch sequencing on the
// context's stream, and result read-back.
#include <algorithm>
#include <array>
#include <map>
#include <chrono>
#include <random>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pm.h"
#include "pm_internal.h"

using namespace pm;

// Device and pinned buffers a launch sequence runs in: the context's own
// (grown as calls need) or a batch's (sized once when the batch is made).
struct Workspace {
    uint8_t* arena = nullptr;
    size_t arena_cap = 0;
    uint8_t* slots = nullptr;   // per-group global slots
    size_t slots_cap = 0;
    uint8_t* pinned = nullptr;  // read-back of statistics, counters, status
    size_t pinned_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;  // prepare | trajectories
    void release()
    {
        if (arena) cudaFree(arena);
        if (slots) cudaFree(slots);
        if (pinned) cudaFreeHost(pinned);
        if (ev0) { cudaEventDestroy(ev0); cudaEventDestroy(ev1); cudaEventDestroy(ev2); }
        *this = Workspace{};
    }
};

struct pm_batch;

struct pm_context {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int sm_count = 0;
    std::string last_error;
    Workspace ws;
    Workspace ws2;                // the rounds of a call with an RSE target or a time budget
    int* cancel_host = nullptr;   // cancel flag: pinned host word mapped into the device
    int* cancel_dev = nullptr;
    std::map<std::string, std::array<int, 6>> tuned;  // autotuned layout policy per size class
    std::vector<pm_batch*> batches;                     // live batches (destroyed with the context)
    double last_traj_ms = 0, last_prep_ms = 0, last_grad_ms = 0;
    uint64_t last_h2d = 0, last_d2h = 0;
    int last_grid = 0, last_wpc = 0;
    Plan last_plan{};
};

namespace {

pm_status fail(pm_context* ctx, pm_status st, const std::string& msg)
{
    if (ctx) ctx->last_error = msg;
    return st;
}

#define PM_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

pm_status grow(pm_context* ctx, uint8_t** buf, size_t* cap, size_t need)
{
    if (need <= *cap) return PM_OK;
    if (*buf) {
        PM_CUDA(cudaStreamSynchronize(ctx->stream));
        PM_CUDA(cudaFree(*buf));
        *buf = nullptr;
        *cap = 0;
    }
    size_t c = need + need / 4;
    PM_CUDA(cudaMalloc(buf, c));
    *cap = c;
    return PM_OK;
}

pm_status grow_pinned(pm_context* ctx, Workspace& ws, size_t need)
{
    if (need <= ws.pinned_cap) return PM_OK;
    if (ws.pinned) {
        PM_CUDA(cudaStreamSynchronize(ctx->stream));
        PM_CUDA(cudaFreeHost(ws.pinned));
        ws.pinned = nullptr;
        ws.pinned_cap = 0;
    }
    PM_CUDA(cudaMallocHost(&ws.pinned, need));
    ws.pinned_cap = need;
    return PM_OK;
}

// a device allocation freed when it goes out of scope
struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

// bump layout over the arena (256-byte aligned pieces)
struct Layout {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        const size_t p = off;
        off = align_up(off + (bytes ? bytes : 1), 256);
        return p;
    }
};

pm_status check_schedule(pm_context* ctx, const pm_schedule* s)
{
    if (!s) return fail(ctx, PM_EINVAL, "schedule is NULL");
    if (s->vertex_rule < 0 || s->vertex_rule > 1) return fail(ctx, PM_EINVAL, "bad vertex_rule");
    if (s->sk < 0 || s->sk > 3) return fail(ctx, PM_EINVAL, "bad sk policy");
    if (s->dm < 0 || s->dm > 3) return fail(ctx, PM_EINVAL, "bad dm policy");
    if (s->precision < 0 || s->precision > 1) return fail(ctx, PM_EINVAL, "bad precision");
    if (s->K0 < 0 || s->K < 0 || s->local_cap < 0) return fail(ctx, PM_EINVAL, "bad K0/K/local_cap");
    if (!(s->theta == s->theta)) return fail(ctx, PM_EINVAL, "theta is NaN");
    if (!(s->rse_target >= 0 && s->rse_target < INFINITY)) return fail(ctx, PM_EINVAL, "bad rse_target");
    if (!(s->time_budget_s >= 0 && s->time_budget_s < INFINITY)) return fail(ctx, PM_EINVAL, "bad time_budget_s");
    if (s->learned && (s->sk != 0 || s->precision != 0))
        return fail(ctx, PM_EINVAL, "the learned proposal needs sk = NONE and the FP32 proposal");
    return PM_OK;
}

pm_status check_csr(pm_context* ctx, const pm_csr* c)
{
    if (!c) return fail(ctx, PM_EINVAL, "csr is NULL");
    if (c->n < 1) return fail(ctx, PM_EINVAL, "n must be >= 1");
    if (c->n > kMaxN) return fail(ctx, PM_EUNSUPPORTED, "n above the supported maximum (2^22)");
    if (c->nnz < 0 || c->nnz >= ((int64_t)1 << 31)) return fail(ctx, PM_EINVAL, "bad nnz");
    if (!c->row_ptr || (c->nnz > 0 && !c->col_idx)) return fail(ctx, PM_EINVAL, "NULL csr array");
    if (c->on_device != 0 && c->on_device != 1) return fail(ctx, PM_EINVAL, "bad on_device");
    if (!c->on_device) {  // cheap host-side checks; the device re-validates everything
        if (c->row_ptr[0] != 0 || c->row_ptr[c->n] != c->nnz) return fail(ctx, PM_EINVAL, "row_ptr ends");
    }
    return PM_OK;
}

}  // namespace

struct pm_model {
    int device = 0;
    float* master = nullptr;  // FP32 parameters [4801]
    float* m1 = nullptr;      // Adam first moment
    float* m2 = nullptr;      // Adam second moment
    float* grad = nullptr;
    void* img = nullptr;      // BF16 device image (DevModel)
    int step = 0;
};

namespace {

// Layout policy of one matrix: which of the plan's choices to take.  The
// heuristic below and the autotuner (pm_batch_create) both produce a policy;
// plan_for() turns it into a Plan for a given matrix and shared-memory budget.
struct Policy {
    int staged = 0, rc_smem = 0, gstate = 0, g = 1, dm_smem = 0, pair = 0;
    bool operator==(const Policy& o) const
    {
        return staged == o.staged && rc_smem == o.rc_smem && gstate == o.gstate && g == o.g && dm_smem == o.dm_smem &&
               pair == o.pair;
    }
    std::array<int, 6> key() const { return {staged, rc_smem, gstate, g, dm_smem, pair}; }
    static Policy of_key(const std::array<int, 6>& k)
    {
        Policy p;
        p.staged = k[0]; p.rc_smem = k[1]; p.gstate = k[2]; p.g = k[3]; p.dm_smem = k[4]; p.pair = k[5];
        return p;
    }
};

// schedules a pair plan can run: no inner SK, DM or Local repair
bool pair_schedule(const Sched& s) { return s.sk == 0 && s.dm == 0; }

// trajectories the GPU runs at once in the usual layouts: one per warp of
// every SM, two per warp for the schedules the pair layout serves
uint64_t traj_slots(const pm_context* ctx, const Sched& s)
{
    return (uint64_t)ctx->sm_count * kCtaWarps * (pair_schedule(s) ? 2u : 1u);
}

int learned_smem(bool learned) { return learned ? (model_infer_bytes() + 15) / 16 * 16 : 0; }

// Plan of one matrix under a policy, or groups = 0 if it does not fit.
Plan plan_for(int n, int64_t m, int rb, const Sched& s, int smem_max, bool learned, const Policy& pol)
{
    const bool full = s.sk == 1 || s.sk == 2;
    const bool need_rc = s.sk != 0;
    const bool dm = s.dm != 0;
    const int avail = smem_max - kCtaMiscBytes - learned_smem(learned);
    Plan p{};
    if (pol.pair) {  // two trajectories per warp, state in shared memory
        if (!pair_schedule(s) || pol.g != 1 || pol.gstate || pol.rc_smem || pol.dm_smem || (pol.staged && n > 65535))
            return p;
        p.g = 1;
        p.pair = 1;
        p.staged = pol.staged;
        p.mat_bytes = pol.staged ? staged_matrix_bytes(n, m, false) : 0;
        if (p.mat_bytes >= avail) return p;
        p.state_bytes = pair_state_bytes(n, learned);
        p.groups = std::min((avail - p.mat_bytes) / p.state_bytes, 2 * pair_cta_warps(learned)) & ~1;
        if (p.groups < 0) p.groups = 0;
        return p;
    }
    p.lists = full;
    p.g = pol.g;
    // several warps per trajectory: full-SK schedules, and DM schedules whose
    // state is in global memory (the group runs the DM's component step)
    if (pol.g < 1 || pol.g > kCtaWarps || (pol.g & (pol.g - 1)) || (!full && pol.g != 1 && !(dm && pol.gstate)))
        return p;
    if (pol.gstate) {
        p.gstate = 1;
        p.rc_smem = need_rc;
        p.state_bytes = kGroupMiscInts * 4 + (learned ? 32 * 24 * 2 : 0);
        p.mat_bytes = 0;
        p.groups = kCtaWarps / p.g;
        if (p.groups * p.state_bytes > avail) p.groups = 0;
        return p;
    }
    if ((pol.rc_smem && !need_rc) || (pol.staged && n > 65535) || (pol.dm_smem && !dm)) return p;
    p.staged = pol.staged;
    p.rc_smem = pol.rc_smem;
    p.dm_smem = pol.dm_smem;
    p.mat_bytes = pol.staged ? staged_matrix_bytes(n, m, dm) : 0;
    if (p.mat_bytes >= avail) return p;
    p.state_bytes = group_state_bytes(n, m, rb, pol.rc_smem, full, learned, pol.dm_smem != 0);
    const int fit = (avail - p.mat_bytes) / p.state_bytes;
    p.groups = std::min(fit, kCtaWarps / p.g);
    if (p.groups < 0) p.groups = 0;
    return p;
}

// Candidate policies of a matrix (those whose plan fits), heuristic first.
std::vector<Policy> candidate_policies(int n, int64_t m, int rb, const Sched& s, int smem_max, bool learned)
{
    const bool full = s.sk == 1 || s.sk == 2;
    const bool need_rc = s.sk != 0;
    const bool dm = s.dm != 0;
    std::vector<Policy> out;
    const int combos[4][2] = {{1, 1}, {0, 1}, {1, 0}, {0, 0}};
    for (int g = 1; g <= ((full || dm) ? kCtaWarps : 1); g *= 2) {
        for (int dms = 0; dms <= (dm ? 1 : 0); ++dms) {
            for (const auto& cb : combos) {
                Policy pol;
                pol.staged = cb[0];
                pol.rc_smem = cb[1];
                pol.g = g;
                pol.dm_smem = dms;
                if (pol.rc_smem && !need_rc) continue;
                const Plan p = plan_for(n, m, rb, s, smem_max, learned, pol);
                if (p.groups >= 1 && (p.groups * p.g >= 4 || !full || dms)) out.push_back(pol);
            }
        }
        Policy gs;
        gs.gstate = 1;
        gs.rc_smem = need_rc;
        gs.g = g;
        if (plan_for(n, m, rb, s, smem_max, learned, gs).groups >= 1) out.push_back(gs);
    }
    if (pair_schedule(s)) {
        for (int st = 1; st >= 0; --st) {
            Policy pp;
            pp.pair = 1;
            pp.staged = st;
            if (plan_for(n, m, rb, s, smem_max, learned, pp).groups >= 4) out.push_back(pp);
        }
    }
    return out;
}

// Heuristic plan: schedules without inner SK or DM run two trajectories per
// warp (matrix staged if it fits) when that keeps at least 8 warps busy;
// otherwise matrix and scaling vectors in shared memory if they fit,
// then scaling vectors only, then neither; full-SK schedules spread a
// trajectory over the fewest warps that keep >= 8 warps of the CTA busy,
// other schedules run one warp per trajectory with as many groups as fit; a
// matrix whose state fits fewer than four groups keeps it in global memory.
Plan make_plan(int n, int64_t m, int rb, const Sched& s, int smem_max, bool learned)
{
    const bool full = s.sk == 1 || s.sk == 2;
    const bool need_rc = s.sk != 0;
    if (pair_schedule(s)) {  // two trajectories per warp while at least 8 warps stay busy
        for (int st = 1; st >= 0; --st) {
            Policy pp;
            pp.pair = 1;
            pp.staged = st;
            const Plan p = plan_for(n, m, rb, s, smem_max, learned, pp);
            if (p.groups >= 16) return p;
        }
    }
    Plan best{};
    int best_score = -1;
    const int combos[4][2] = {{1, 1}, {0, 1}, {1, 0}, {0, 0}};
    for (const auto& cb : combos) {
        if (cb[1] && !need_rc) continue;
        Plan chosen{};
        for (int g = 1; g <= (full ? kCtaWarps : 1); g *= 2) {
            Policy pol;
            pol.staged = cb[0];
            pol.rc_smem = cb[1];
            pol.g = g;
            const Plan p = plan_for(n, m, rb, s, smem_max, learned, pol);
            if (p.groups < 1) break;
            chosen = p;
            if (p.groups * g == kCtaWarps) break;
        }
        if (chosen.groups < 1) continue;
        const int busy = chosen.g * chosen.groups;
        const int score = busy >= (full ? 8 : 12) ? 1000 : busy;
        if (score > best_score) {
            best = chosen;
            best_score = score;
            if (score >= 1000) break;
        }
    }
    if (best_score < 4) {  // large n: trajectory state in the group's global slot
        Policy gs;
        gs.gstate = 1;
        gs.rc_smem = need_rc;
        // DM schedules on large matrices: one trajectory per CTA, whose 16 warps
        // share the DM's component step (a warp-serial step over 2n vertices in
        // global memory would dominate)
        gs.g = full ? 4 : (s.dm != 0 && n >= 8192) ? kCtaWarps : 1;
        const Plan p = plan_for(n, m, rb, s, smem_max, learned, gs);
        if (p.groups >= 1) best = p;
    }
    return best;
}

Policy policy_of(const Plan& p)
{
    Policy o;
    o.staged = p.staged; o.rc_smem = p.rc_smem; o.gstate = p.gstate; o.g = p.g; o.dm_smem = p.dm_smem;
    o.pair = p.pair;
    return o;
}

// size class of a matrix for the autotuner: half-octaves of n
int size_class(int n) { return (int)std::floor(2.0 * std::log2((double)std::max(1, n))); }

std::string class_key(int cls, const Sched& s, bool learned)
{
    return std::to_string(cls) + "|" + std::to_string(s.vertex_rule) + std::to_string(s.sk) + std::to_string(s.dm) +
           std::to_string(s.precision) + std::to_string(s.K) + "|" + (learned ? "L" : "-");
}

// The layout of a matrix when the caller gives none: the autotuner's choice
// cached in the context for its size class and schedule, if one fits, else
// the heuristic.
Plan default_plan(const pm_context* ctx, int n, int64_t m, int rb, const Sched& s, int smem_max, bool learned)
{
    auto it = ctx->tuned.find(class_key(size_class(n), s, learned));
    if (it != ctx->tuned.end()) {
        const Policy pol = Policy::of_key(it->second);
        const Plan p = plan_for(n, m, rb, s, smem_max, learned, pol);
        if (p.groups >= 1) return p;
    }
    return make_plan(n, m, rb, s, smem_max, learned);
}

struct Run {
    // inputs
    const pm_csr* mats = nullptr;
    int count = 0;
    std::vector<uint64_t> ntraj;
    uint64_t first_traj = 0;
    uint32_t matrix_index0 = 0;  // matrix index of mats[0] (others: +k)
    uint64_t seed = 0;
    Sched s{};
    bool trace = false;
    bool prep_only = false;
    // host outputs
    pm_result* outs = nullptr;
    int32_t *chosen = nullptr, *deg_v = nullptr, *dead_step = nullptr;
    double* log_x = nullptr;
    float* logits = nullptr;        // trace: [T][n][logit_stride]
    uint32_t logit_stride = 0;
    const void* model = nullptr;    // learned proposal device image
    // recording (device buffers)
    float* rec_feat = nullptr;
    float* rec_target = nullptr;
    unsigned long long* rec_key = nullptr;
    uint32_t* rec_group = nullptr;
    unsigned long long* rec_count = nullptr;
    unsigned long long rec_cap = 0;
    int32_t* ok_out = nullptr;
    uint8_t* keep_out = nullptr;
    double *r_out = nullptr, *c_out = nullptr;
    // matrices already prepared in device memory that outlives the run
    // (host copies of their descriptors; mats then supply n and nnz only)
    const DevMatrix* prepared = nullptr;
    // per matrix, the local index of its first trajectory (empty: 0)
    std::vector<uint64_t> first_local;
    // order of the matrices' chunks in the launch (empty: most expensive first)
    std::vector<int> order;
    // run control (0: none): device-side time budget of the trajectory launch
    uint64_t budget_ns = 0;
    double rse_target = 0, budget_s = 0;
};

struct MatOff {
    size_t rp64, ci_in, val_in, a_rp, a_ci, a_val, a_cp, a_ri, a_ce, keep, rp, ci, rv, cp, ri, cv, ce, r0, c0, deg0,
        tree0, dmws;
};

// Everything the launch sequence of a Run needs, laid out in a workspace.
struct Staged {
    bool fp64 = false;
    size_t rb = 4;
    int n_max = 1;
    int64_t m_max = 1;
    std::vector<uint64_t> prefix;
    uint64_t total = 0;
    std::vector<MatOff> mo;
    size_t o_mats = 0, o_inputs = 0, o_prefix = 0, o_logx = 0, o_counters = 0, o_work = 0, o_status = 0;
    size_t o_parts = 0, o_sout = 0, o_chosen = 0, o_degv = 0, o_dead = 0, o_logits = 0;
    size_t o_plans = 0, o_chunks = 0, o_cctr = 0, o_tstart = 0, layout_end = 0, chunk_cap = 0;
    uint32_t stop_bits = 0;       // ST_TIMEOUT / ST_CANCELLED seen by collect()
    int chunks_stats = 1;
    int cta_warps = kCtaWarps;    // warps per CTA of the trajectory launch
    std::vector<Plan> plans;
    std::vector<Chunk> chunks;
    int smem_need = kCtaMiscBytes;
    int grid = 0;
    TrajParams tp{};
    uint64_t h2d = 0, d2h = 0;
    bool launch_traj = false;
    // pinned read-back
    StatsOut* h_sout = nullptr;
    unsigned long long* h_cnt = nullptr;
    uint32_t* h_status = nullptr;
    DevMatrix* h_mats = nullptr;
};

// Phase 1: arena layout, inputs and matrix descriptors (uploads on the stream).
pm_status stage_inputs(pm_context* ctx, Workspace& ws, const Run& R, Staged& S, size_t min_chunks = 0)
{
    const int count = R.count;
    S.fp64 = R.s.precision == 1;
    S.rb = S.fp64 ? 8 : 4;
    S.n_max = 1;
    S.m_max = 1;
    for (int k = 0; k < count; ++k) {
        S.n_max = std::max(S.n_max, R.mats[k].n);
        S.m_max = std::max<int64_t>(S.m_max, R.mats[k].nnz);
    }
    S.prefix.assign(count + 1, 0);
    for (int k = 0; k < count; ++k) S.prefix[k + 1] = S.prefix[k] + R.ntraj[k];
    S.total = S.prefix[count];
    const size_t rb = S.rb;

    Layout L;
    S.mo.resize(R.prepared ? 0 : count);
    for (int k = 0; k < count && !R.prepared; ++k) {
        const pm_csr& c = R.mats[k];
        const int n = c.n;
        const size_t m = (size_t)c.nnz;
        const bool w = c.values != nullptr;
        MatOff& o = S.mo[k];
        o.rp64 = c.on_device ? 0 : L.take((n + 1) * 8);
        o.ci_in = c.on_device ? 0 : L.take(m * 4);
        o.val_in = (c.on_device || !w) ? 0 : L.take(m * 4);
        o.a_rp = L.take((n + 1) * 4);
        o.a_ci = L.take(m * 4);
        o.a_val = w ? L.take(m * 4) : 0;
        o.a_cp = L.take((n + 1) * 4);
        o.a_ri = L.take(m * 4);
        o.a_ce = L.take(m * 4);
        o.keep = L.take(m);
        o.rp = L.take((n + 1) * 4);
        o.ci = L.take(m * 4);
        o.rv = w ? L.take(m * 4) : 0;
        o.cp = L.take((n + 1) * 4);
        o.ri = L.take(m * 4);
        o.cv = w ? L.take(m * 4) : 0;
        o.ce = L.take(m * 4);
        o.r0 = L.take(n * rb);
        o.c0 = L.take(n * rb);
        o.deg0 = L.take((size_t)((2 * n + 7) & ~7) * 2);
        o.tree0 = L.take((size_t)std::max(1, tree_geom(n).total) * 4);
        o.dmws = L.take((size_t)dm_ws_ints(n) * 4);
    }
    S.o_mats = L.take(sizeof(DevMatrix) * count);
    S.o_inputs = L.take(sizeof(DevInput) * count);
    S.o_prefix = L.take(8 * (count + 1));
    S.o_logx = L.take(8 * std::max<uint64_t>(S.total, 1));
    S.o_counters = L.take(8 * kCounters * count);
    S.o_work = L.take(8);
    S.o_status = L.take(4);
    uint64_t max_t = 1;
    for (int k = 0; k < count; ++k) max_t = std::max(max_t, R.ntraj[k]);
    S.chunks_stats = (int)std::min<uint64_t>(1024, std::max<uint64_t>(1, max_t / 16384));
    S.o_parts = L.take(sizeof(StatsPartial) * (size_t)count * S.chunks_stats);
    S.o_sout = L.take(sizeof(StatsOut) * count);
    if (R.trace) {
        S.o_chosen = L.take(4 * S.total * 2 * (size_t)S.n_max);
        S.o_degv = L.take(4 * S.total * (size_t)S.n_max);
        S.o_dead = L.take(4 * std::max<uint64_t>(S.total, 1));
        if (R.model && R.logit_stride) S.o_logits = L.take(4 * S.total * (size_t)S.n_max * R.logit_stride);
    }
    // the plans and the chunk list (a chunk holds 2 x groups >= 2 trajectories)
    S.chunk_cap = std::max<size_t>(S.total / 2 + 2 * (size_t)count, min_chunks);
    S.o_plans = L.take(sizeof(Plan) * count);
    S.o_chunks = L.take(sizeof(Chunk) * S.chunk_cap);
    S.o_cctr = L.take(8);
    S.o_tstart = L.take(8);
    S.layout_end = L.off;
    pm_status st = grow(ctx, &ws.arena, &ws.arena_cap, L.off);
    if (st != PM_OK) return st;
    uint8_t* A = ws.arena;
    auto P = [&](size_t off) { return (void*)(A + off); };

    std::vector<DevMatrix> hm(count);
    std::vector<DevInput> hi(count);
    if (R.prepared) std::copy(R.prepared, R.prepared + count, hm.begin());
    for (int k = 0; k < count && !R.prepared; ++k) {
        const pm_csr& c = R.mats[k];
        const MatOff& o = S.mo[k];
        const int n = c.n;
        const size_t m = (size_t)c.nnz;
        DevInput& I = hi[k];
        I.n = n;
        I.m = (int)m;
        if (!c.on_device) S.h2d += (n + 1) * 8 + m * 4 + (c.values ? m * 4 : 0);
        if (c.on_device) {
            I.rp64 = c.row_ptr;
            I.ci_in = c.col_idx;
            I.val_in = c.values;
        } else {
            PM_CUDA(cudaMemcpyAsync(P(o.rp64), c.row_ptr, (n + 1) * 8, cudaMemcpyHostToDevice, ctx->stream));
            if (m) PM_CUDA(cudaMemcpyAsync(P(o.ci_in), c.col_idx, m * 4, cudaMemcpyHostToDevice, ctx->stream));
            if (c.values && m)
                PM_CUDA(cudaMemcpyAsync(P(o.val_in), c.values, m * 4, cudaMemcpyHostToDevice, ctx->stream));
            I.rp64 = (const int64_t*)P(o.rp64);
            I.ci_in = (const int32_t*)P(o.ci_in);
            I.val_in = c.values ? (const float*)P(o.val_in) : nullptr;
        }
        DevMatrix& M = hm[k];
        std::memset(&M, 0, sizeof(M));
        M.n = n;
        M.m_a = (int)m;
        M.idx = (int)(R.matrix_index0 + (uint32_t)k);
        const bool w = c.values != nullptr;
        M.a_rp = (int*)P(o.a_rp); M.a_ci = (int*)P(o.a_ci); M.a_val = w ? (float*)P(o.a_val) : nullptr;
        M.a_cp = (int*)P(o.a_cp); M.a_ri = (int*)P(o.a_ri); M.a_ce = (int*)P(o.a_ce);
        M.keep = (uint8_t*)P(o.keep);
        M.rp = (int*)P(o.rp); M.ci = (int*)P(o.ci); M.rv = w ? (float*)P(o.rv) : nullptr;
        M.cp = (int*)P(o.cp); M.ri = (int*)P(o.ri); M.cv = w ? (float*)P(o.cv) : nullptr; M.ce = (int*)P(o.ce);
        M.r0 = P(o.r0); M.c0 = P(o.c0);
        M.deg0 = (uint16_t*)P(o.deg0);
        M.tree0 = (uint32_t*)P(o.tree0);
        M.dm_ws = (int*)P(o.dmws);
    }
    PM_CUDA(cudaMemcpyAsync(P(S.o_mats), hm.data(), sizeof(DevMatrix) * count, cudaMemcpyHostToDevice, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(P(S.o_inputs), hi.data(), sizeof(DevInput) * count, cudaMemcpyHostToDevice, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(P(S.o_prefix), S.prefix.data(), 8 * (count + 1), cudaMemcpyHostToDevice, ctx->stream));
    S.h2d += sizeof(DevMatrix) * count + sizeof(DevInput) * count + 8 * (count + 1);

    // pinned read-back area
    const size_t pin_need = sizeof(StatsOut) * count + 8 * kCounters * count + 8 + sizeof(DevMatrix) * count + 128;
    st = grow_pinned(ctx, ws, pin_need);
    if (st != PM_OK) return st;
    S.h_sout = (StatsOut*)ws.pinned;
    S.h_cnt = (unsigned long long*)(S.h_sout + count);
    S.h_status = (uint32_t*)(S.h_cnt + kCounters * count);
    S.h_mats = (DevMatrix*)(ws.pinned + align_up(sizeof(StatsOut) * count + 8 * kCounters * count + 8, 64));
    if (!ws.ev0) {
        PM_CUDA(cudaEventCreate(&ws.ev0));
        PM_CUDA(cudaEventCreate(&ws.ev1));
        PM_CUDA(cudaEventCreate(&ws.ev2));
    }
    return PM_OK;
}

// Phase 2: plans (heuristic, or the given ones), chunk list, slots and the
// trajectory kernel's parameters.
pm_status stage_plans(pm_context* ctx, Workspace& ws, const Run& R, Staged& S, const std::vector<Plan>* given)
{
    const int count = R.count;
    S.launch_traj = !R.prep_only && S.total > 0;
    if (!S.launch_traj) return PM_OK;
    uint8_t* A = ws.arena;
    auto P = [&](size_t off) { return (void*)(A + off); };
    const bool scales = R.s.sk != 0;
    const bool local = R.s.sk == 3;
    const bool dm = R.s.dm != 0;
    const int smem_max = traj_max_smem_bytes();
    if (smem_max <= 0) return fail(ctx, PM_ECUDA, "cannot query the shared-memory limit");
    S.plans.assign(count, Plan{});
    S.smem_need = kCtaMiscBytes;
    for (int k = 0; k < count; ++k) {
        S.plans[k] = given ? (*given)[k] : default_plan(ctx, R.mats[k].n, R.mats[k].nnz, (int)S.rb, R.s, smem_max,
                                                         R.model != nullptr);
        if (S.plans[k].pair && (R.trace || R.rec_feat)) {  // traces and recordings run one trajectory per warp
            Policy pol = policy_of(S.plans[k]);
            pol.pair = 0;
            S.plans[k] = plan_for(R.mats[k].n, R.mats[k].nnz, (int)S.rb, R.s, smem_max, R.model != nullptr, pol);
        }
        if (S.plans[k].groups < 1)
            return fail(ctx, PM_EUNSUPPORTED, "trajectory state does not fit in shared memory");
        S.smem_need = std::max(S.smem_need, kCtaMiscBytes + learned_smem(R.model != nullptr) + S.plans[k].mat_bytes +
                                                S.plans[k].groups * S.plans[k].state_bytes);
    }
    size_t gstate_bytes = 0;
    for (int k = 0; k < count; ++k)
        if (S.plans[k].gstate)
            gstate_bytes = std::max(gstate_bytes, global_state_bytes(R.mats[k].n, (int)S.rb, S.plans[k].lists != 0));
    const SlotLayout sl =
        slot_layout(S.n_max, (int)S.m_max, (int)S.rb, scales, local, dm, gstate_bytes, R.model != nullptr);
    // chunks: the caller's order, else the most expensive matrices first; a
    // few trajectories per group
    std::vector<int> order(count);
    for (int k = 0; k < count; ++k) order[k] = k;
    const bool full_sk = R.s.sk == 1 || R.s.sk == 2;
    if ((int)R.order.size() == count) {
        order = R.order;
    } else {
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const double ca = (double)R.mats[a].nnz * (full_sk ? R.mats[a].n : 1);
            const double cb = (double)R.mats[b].nnz * (full_sk ? R.mats[b].n : 1);
            return ca > cb;
        });
    }
    S.chunks.clear();
    for (int k : order) {
        const uint64_t csz = (uint64_t)S.plans[k].groups * 2;
        const uint64_t base = R.first_local.empty() ? 0 : R.first_local[k];
        for (uint64_t f = 0; f < R.ntraj[k]; f += csz) {
            Chunk c;
            c.k = k;
            c.first = base + f;
            c.slot0 = S.prefix[k] + f;
            c.count = (uint32_t)std::min<uint64_t>(csz, R.ntraj[k] - f);
            S.chunks.push_back(c);
        }
    }
    if (S.chunks.size() > S.chunk_cap) return fail(ctx, PM_EINVAL, "internal: chunk list");
    S.grid = ctx->sm_count;
    PM_CUDA(cudaMemcpyAsync(P(S.o_plans), S.plans.data(), sizeof(Plan) * count, cudaMemcpyHostToDevice, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(P(S.o_chunks), S.chunks.data(), sizeof(Chunk) * S.chunks.size(), cudaMemcpyHostToDevice,
                            ctx->stream));
    S.h2d += sizeof(Plan) * count + sizeof(Chunk) * S.chunks.size();
    // every plan with trajectories a pair plan: the 768-thread pair-only kernel
    bool all_pair = true;
    for (int k = 0; k < count; ++k)
        if (R.ntraj[k] > 0 && !S.plans[k].pair) all_pair = false;
    S.cta_warps = all_pair ? pair_cta_warps(R.model != nullptr) : kCtaWarps;
    const size_t need_slots = sl.bytes * (size_t)S.grid * S.cta_warps;
    pm_status st = grow(ctx, &ws.slots, &ws.slots_cap, need_slots);
    if (st != PM_OK) return st;
    TrajParams& tp = S.tp;
    tp = TrajParams{};
    tp.mats = (const DevMatrix*)P(S.o_mats);
    tp.plans = (const Plan*)P(S.o_plans);
    tp.chunks = (const Chunk*)P(S.o_chunks);
    tp.n_chunks = (int)S.chunks.size();
    tp.count = count;
    tp.n_max = S.n_max;
    tp.prefix = (const uint64_t*)P(S.o_prefix);
    tp.first_traj = R.first_traj;
    tp.seed = R.seed;
    tp.s = R.s;
    tp.log_x = (double*)P(S.o_logx);
    tp.counters = (unsigned long long*)P(S.o_counters);
    tp.chunk_counter = (int*)P(S.o_cctr);
    tp.status = (uint32_t*)P(S.o_status);
    tp.slots = ws.slots;
    tp.slot = sl;
    tp.cta_warps = S.cta_warps;
    tp.pair_kernel = (all_pair && R.model == nullptr) ? 1 : 0;
    if (R.trace) {
        tp.chosen = (int32_t*)P(S.o_chosen);
        tp.deg_v = (int32_t*)P(S.o_degv);
        tp.dead_step = (int32_t*)P(S.o_dead);
        if (R.model && R.logit_stride) {
            tp.trace_logits = (float*)P(S.o_logits);
            tp.logit_stride = (int)R.logit_stride;
        }
    }
    tp.budget_ns = R.budget_ns;
    tp.hard_ns = R.budget_ns ? 2 * R.budget_ns + 5000000000ull : 0;
    tp.t_start = (unsigned long long*)P(S.o_tstart);
    tp.cancel = ctx->cancel_dev;
    tp.model = R.model;
    tp.rec_feat = R.rec_feat;
    tp.rec_target = R.rec_target;
    tp.rec_key = R.rec_key;
    tp.rec_group = R.rec_group;
    tp.rec_count = R.rec_count;
    tp.rec_cap = R.rec_cap;
    return PM_OK;
}

// Phase 3: the launch sequence of one run on the stream, in three segments
// (each capturable: its host sources and destinations live in the workspace):
// preprocessing, the trajectory kernel, statistics and read-back.
// NVTX range over a scope (named phases for profilers: `ncu --nvtx
// --nvtx-include "pm trajectories/"` selects the trajectory launches)
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};

pm_status enqueue_prep(pm_context* ctx, Workspace& ws, const Run& R, Staged& S)
{
    NvtxScope nv("pm preprocess");
    uint8_t* A = ws.arena;
    auto P = [&](size_t off) { return (void*)(A + off); };
    PM_CUDA(cudaMemsetAsync(P(S.o_counters), 0, 8 * kCounters * R.count, ctx->stream));
    PM_CUDA(cudaMemsetAsync(P(S.o_work), 0, 8, ctx->stream));
    PM_CUDA(cudaMemsetAsync(P(S.o_status), 0, 4, ctx->stream));
    if (!R.prepared)
        PM_CUDA(launch_prepare((DevMatrix*)P(S.o_mats), (const DevInput*)P(S.o_inputs), R.count, R.s, S.m_max, S.n_max,
                               (uint32_t*)P(S.o_status), ctx->stream));
    return PM_OK;
}

pm_status enqueue_traj(pm_context* ctx, Workspace& ws, const Run& R, Staged& S)
{
    if (!S.launch_traj) return PM_OK;
    NvtxScope nv("pm trajectories");
    PM_CUDA(cudaMemsetAsync(ws.arena + S.o_cctr, 0, 8, ctx->stream));
    PM_CUDA(cudaMemsetAsync(ws.arena + S.o_tstart, 0, 8, ctx->stream));
    // ln X = NaN (all bits set) marks trajectories a stopped launch never started
    PM_CUDA(cudaMemsetAsync(ws.arena + S.o_logx, 0xFF, 8 * S.total, ctx->stream));
    if (S.tp.trace_logits)
        PM_CUDA(cudaMemsetAsync(S.tp.trace_logits, 0, 4 * S.total * (size_t)S.n_max * R.logit_stride,
                                ctx->stream));
    PM_CUDA(launch_trajectories(S.tp, S.grid, S.smem_need, R.trace, ctx->stream));
    return PM_OK;
}

pm_status enqueue_tail(pm_context* ctx, Workspace& ws, const Run& R, Staged& S)
{
    NvtxScope nv("pm statistics");
    const int count = R.count;
    uint8_t* A = ws.arena;
    auto P = [&](size_t off) { return (void*)(A + off); };
    if (S.launch_traj) {
        PM_CUDA(launch_stats((const double*)P(S.o_logx), S.prefix.data(), (const uint64_t*)P(S.o_prefix), count,
                             (StatsPartial*)P(S.o_parts), S.chunks_stats, (StatsOut*)P(S.o_sout), ctx->stream));
        PM_CUDA(cudaMemcpyAsync(S.h_sout, P(S.o_sout), sizeof(StatsOut) * count, cudaMemcpyDeviceToHost, ctx->stream));
        PM_CUDA(cudaMemcpyAsync(S.h_cnt, P(S.o_counters), 8 * kCounters * count, cudaMemcpyDeviceToHost, ctx->stream));
    }
    PM_CUDA(cudaMemcpyAsync(S.h_status, P(S.o_status), 4, cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(S.h_mats, P(S.o_mats), sizeof(DevMatrix) * count, cudaMemcpyDeviceToHost, ctx->stream));
    return PM_OK;
}

// the three segments with the timing events between them
pm_status enqueue(pm_context* ctx, Workspace& ws, const Run& R, Staged& S)
{
    PM_CUDA(cudaEventRecord(ws.ev2, ctx->stream));
    pm_status st = enqueue_prep(ctx, ws, R, S);
    if (st != PM_OK) return st;
    PM_CUDA(cudaEventRecord(ws.ev0, ctx->stream));
    st = enqueue_traj(ctx, ws, R, S);
    if (st != PM_OK) return st;
    PM_CUDA(cudaEventRecord(ws.ev1, ctx->stream));
    return enqueue_tail(ctx, ws, R, S);
}

// Phase 4 (after the stream synchronised): errors, timings, outputs.
pm_status collect(pm_context* ctx, Workspace& ws, const Run& R, Staged& S, double secs)
{
    const int count = R.count;
    uint8_t* A = ws.arena;
    auto P = [&](size_t off) { return (void*)(A + off); };
    uint64_t d2h = 4 + sizeof(DevMatrix) * count;
    if (S.launch_traj) d2h += sizeof(StatsOut) * count + 8 * kCounters * count;
    {
        float ms = 0;
        ctx->last_prep_ms = (cudaEventElapsedTime(&ms, ws.ev2, ws.ev0) == cudaSuccess) ? ms : -1.0;
        ctx->last_traj_ms = 0;
        if (S.launch_traj) ctx->last_traj_ms = (cudaEventElapsedTime(&ms, ws.ev0, ws.ev1) == cudaSuccess) ? ms : -1.0;
        cudaGetLastError();  // a timing that could not be taken is reported as -1
    }
    ctx->last_grid = S.launch_traj ? S.grid : 0;
    ctx->last_wpc = S.launch_traj ? S.cta_warps : 0;
    ctx->last_plan = (S.launch_traj && !S.plans.empty()) ? S.plans[0] : Plan{};
    const uint32_t status = *S.h_status & ~kStatusStopBits;
    S.stop_bits = *S.h_status & kStatusStopBits;
    if (status & ST_BAD_INPUT) return fail(ctx, PM_EINVAL, "malformed CSR (device validation)");
    if (status & ST_CAPACITY) return fail(ctx, PM_EUNSUPPORTED, "a row or column holds more than 65534 entries");
    if (status) return fail(ctx, PM_EDEVICE, "device status " + std::to_string(status));
    if (const unsigned int hits = traj_bounds_hits())  // PM_DEBUG builds only
        return fail(ctx, PM_EDEVICE, "device bounds check: " + std::to_string(hits) + " out-of-range accesses");

    if (R.trace) {
        const size_t T = S.total, n = R.mats[0].n;
        if (R.chosen) PM_CUDA(cudaMemcpy(R.chosen, P(S.o_chosen), 4 * T * 2 * n, cudaMemcpyDeviceToHost));
        if (R.deg_v) PM_CUDA(cudaMemcpy(R.deg_v, P(S.o_degv), 4 * T * n, cudaMemcpyDeviceToHost));
        if (R.dead_step) PM_CUDA(cudaMemcpy(R.dead_step, P(S.o_dead), 4 * T, cudaMemcpyDeviceToHost));
        if (R.logits && R.model && R.logit_stride)
            PM_CUDA(cudaMemcpy(R.logits, P(S.o_logits), 4 * T * n * R.logit_stride, cudaMemcpyDeviceToHost));
    }
    if (R.log_x && S.total) {
        PM_CUDA(cudaMemcpy(R.log_x, P(S.o_logx), 8 * S.total, cudaMemcpyDeviceToHost));
        d2h += 8 * S.total;
    }
    if (R.prep_only) {
        const pm_csr& c = R.mats[0];
        const size_t rb = S.rb;
        if (R.ok_out) *R.ok_out = S.h_mats[0].ok;
        if (R.keep_out && c.nnz) PM_CUDA(cudaMemcpy(R.keep_out, P(S.mo[0].keep), c.nnz, cudaMemcpyDeviceToHost));
        if (R.r_out || R.c_out) {
            std::vector<uint8_t> tmp((size_t)c.n * rb * 2);
            PM_CUDA(cudaMemcpy(tmp.data(), P(S.mo[0].r0), c.n * rb, cudaMemcpyDeviceToHost));
            PM_CUDA(cudaMemcpy(tmp.data() + c.n * rb, P(S.mo[0].c0), c.n * rb, cudaMemcpyDeviceToHost));
            for (int q = 0; q < c.n; ++q) {
                const double rv = S.fp64 ? ((double*)tmp.data())[q] : (double)((float*)tmp.data())[q];
                const double cv = S.fp64 ? ((double*)(tmp.data() + c.n * rb))[q]
                                         : (double)((float*)(tmp.data() + c.n * rb))[q];
                if (R.r_out) R.r_out[q] = rv;
                if (R.c_out) R.c_out[q] = cv;
            }
        }
    }
    ctx->last_h2d = S.h2d;
    ctx->last_d2h = d2h;
    if (R.outs) {
        double ns_total = 0;
        for (int k = 0; k < count; ++k) ns_total += (double)S.h_cnt[kCounters * k + 5];
        for (int k = 0; k < count; ++k) {
            pm_result& o = R.outs[k];
            std::memset(&o, 0, sizeof(o));
            const StatsOut& so = S.h_sout[k];
            o.log_estimate = so.log_estimate;
            o.estimate = std::exp(so.log_estimate);
            o.ess = so.ess;
            o.p_match = so.p_match;
            o.rel_spread = so.rel_spread;
            o.rse = so.rse;
            o.log_sum_x = so.log_sum_x;
            o.log_sum_x2 = so.log_sum_x2;
            o.n_traj = so.n;
            o.n_alive = so.alive;
            o.n_dm_calls = S.h_cnt[kCounters * k + 0];
            o.n_full_sk = S.h_cnt[kCounters * k + 1];
            o.n_local_sk = S.h_cnt[kCounters * k + 2];
            o.alg_bytes = S.h_cnt[kCounters * k + 3];
            o.mlp_rows = S.h_cnt[kCounters * k + 4];
            o.traj_ns = S.h_cnt[kCounters * k + 5];
            o.kernel_ms = ctx->last_traj_ms;
            o.seconds = secs;
            o.dev_ms = (ns_total > 0 && ctx->last_traj_ms > 0)
                           ? ctx->last_traj_ms * (double)o.traj_ns / ns_total : 0.0;
            o.rounds = 1;
            o.stop = (S.stop_bits & ST_CANCELLED) ? PM_STOP_CANCELLED
                     : (S.stop_bits & ST_TIMEOUT) ? PM_STOP_TIME : PM_STOP_COMPLETE;
        }
    }
    return PM_OK;
}

// status of a call whose launch may have stopped early: outputs are written
pm_status stop_status(pm_context* ctx, uint32_t stop_bits)
{
    if (stop_bits & ST_CANCELLED) return fail(ctx, PM_ECANCELLED, "cancelled (pm_context_cancel)");
    if (stop_bits & ST_TIMEOUT) return fail(ctx, PM_ETIMEOUT, "the time budget ran out");
    return PM_OK;
}

pm_status execute(pm_context* ctx, Run& R)
{
    const auto t0 = std::chrono::steady_clock::now();
    PM_CUDA(cudaSetDevice(ctx->device));
    Staged S;
    ctx->last_traj_ms = ctx->last_prep_ms = 0;
    ctx->last_grid = ctx->last_wpc = 0;
    pm_status st = stage_inputs(ctx, ctx->ws, R, S);
    if (st != PM_OK) return st;
    st = stage_plans(ctx, ctx->ws, R, S, nullptr);
    if (st != PM_OK) return st;
    st = enqueue(ctx, ctx->ws, R, S);
    if (st != PM_OK) return st;
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    st = collect(ctx, ctx->ws, R, S, secs);
    if (st != PM_OK) return st;
    return stop_status(ctx, S.stop_bits);
}

}  // namespace

// Sufficient statistics of disjoint trajectory sets of one matrix (Sec. 2:
// the estimate, ESS and p_match; Sec. 4 "Metrics": relative spread and RSE
// all follow from M, #alive, ln sum X and ln sum X^2), plus the operation
// counts; merged exactly in any order.
struct Suff {
    uint64_t n = 0, alive = 0, n_dm = 0, n_full = 0, n_loc = 0, alg = 0, mlp = 0, traj_ns = 0;
    double lse1 = -INFINITY, lse2 = -INFINITY, kernel_ms = 0, seconds = 0, dev_ms = 0;
    uint32_t rounds = 0;
    static double lse_add(double a, double b)
    {
        if (a == -INFINITY) return b;
        if (b == -INFINITY) return a;
        const double m = a > b ? a : b;
        return m + std::log(std::exp(a - m) + std::exp(b - m));
    }
    void add(const pm_result& o)
    {
        n += o.n_traj;
        alive += o.n_alive;
        if (o.n_alive) {
            lse1 = lse_add(lse1, o.log_sum_x);
            lse2 = lse_add(lse2, o.log_sum_x2);
        }
        n_dm += o.n_dm_calls;
        n_full += o.n_full_sk;
        n_loc += o.n_local_sk;
        alg += o.alg_bytes;
        mlp += o.mlp_rows;
        traj_ns += o.traj_ns;
        dev_ms += o.dev_ms;
        kernel_ms += o.kernel_ms > 0 ? o.kernel_ms : 0;
        seconds += o.seconds > 0 ? o.seconds : 0;
        rounds += o.rounds;
    }
    void fill(pm_result& o) const
    {
        std::memset(&o, 0, sizeof(o));
        o.n_traj = n;
        o.n_alive = alive;
        o.log_sum_x = lse1;
        o.log_sum_x2 = lse2;
        o.n_dm_calls = n_dm;
        o.n_full_sk = n_full;
        o.n_local_sk = n_loc;
        o.alg_bytes = alg;
        o.mlp_rows = mlp;
        o.traj_ns = traj_ns;
        o.dev_ms = dev_ms;
        o.kernel_ms = kernel_ms;
        o.seconds = seconds;
        o.rounds = rounds;
        o.p_match = n ? (double)alive / (double)n : 0.0;
        if (n == 0 || lse1 == -INFINITY) {
            o.log_estimate = -INFINITY;
            o.rel_spread = o.rse = NAN;
            return;
        }
        const double M = (double)n;
        o.log_estimate = lse1 - std::log(M);
        o.estimate = std::exp(o.log_estimate);
        o.ess = std::exp(2 * lse1 - lse2);
        if (n > 1) {  // s_X^2 / mean^2 = (M sum X^2 / (sum X)^2 - 1) M / (M - 1)
            const double ratio = M * std::exp(lse2 - 2 * lse1);
            o.rel_spread = std::sqrt(std::max(0.0, ratio - 1.0) * M / (M - 1.0));
            o.rse = o.rel_spread / std::sqrt(M);
        } else {
            o.rel_spread = o.rse = NAN;
        }
    }
};

namespace {

// Trajectories a matrix must have before its RSE may end its run.
constexpr uint64_t kMinTrajForTarget = 1024;
// Budgeted rounds: the share of the remaining budget one round may plan for
// (the rest is kept for the rounds that follow it, with fresher estimates),
// and the smallest allocation worth a matrix's chunks in a round.
constexpr double kRoundShare = 0.6;
constexpr uint64_t kMinRoundTraj = 256;

// A call with an RSE target or a time budget: preprocessing once, then rounds
// of trajectories over the matrices still running (consecutive trajectory
// ids per matrix, so the rounds together are the trajectories one launch
// would run), statistics merged on the host after each round.  A matrix stops
// when its RSE (Sec. 4 "Metrics") is at most the target with at least
// kMinTrajForTarget trajectories (or all of n_traj) and two alive, or when its
// n_traj ran; the call stops when every matrix has stopped, the budget is
// spent (PM_ETIMEOUT) or the context is cancelled (PM_ECANCELLED).
//
// With an RSE target, a time budget and several matrices, the rounds after
// the first are planned cheapest-to-finish first: each running matrix's trajectories still
// needed for the target (1.1 M (RSE / target)^2 - M) are priced at its
// measured launch time per trajectory in the previous rounds, and the
// matrices are served in increasing order of that price (each round's
// allocation capped at 5x what the matrix has), until the round's plan fills
// kRoundShare of the remaining budget (all of it once little is left).  So
// the budget goes first to the matrices it can bring to the target, and what
// is left to the rest; their chunks run in the same order.
pm_status execute_rounds(pm_context* ctx, Run& R)
{
    const auto t0 = std::chrono::steady_clock::now();
    auto elapsed = [&] { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
    PM_CUDA(cudaSetDevice(ctx->device));
    const int count = R.count;
    // preprocessing (InitialDM, outer SK, degrees, tree) into the context's workspace
    Run Pr;
    Pr.mats = R.mats;
    Pr.count = count;
    Pr.ntraj.assign(count, 0);
    Pr.matrix_index0 = R.matrix_index0;
    Pr.s = R.s;
    Pr.prep_only = true;
    Pr.model = R.model;
    Staged SP;
    pm_status st = stage_inputs(ctx, ctx->ws, Pr, SP);
    if (st == PM_OK) st = stage_plans(ctx, ctx->ws, Pr, SP, nullptr);
    if (st == PM_OK) st = enqueue(ctx, ctx->ws, Pr, SP);
    if (st != PM_OK) return st;
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    st = collect(ctx, ctx->ws, Pr, SP, 0.0);
    if (st != PM_OK) return st;
    const double prep_ms = ctx->last_prep_ms;
    uint64_t h2d = ctx->last_h2d, d2h = ctx->last_d2h;
    std::vector<DevMatrix> dms(SP.h_mats, SP.h_mats + count);
    // rounds
    std::vector<uint64_t> req_prefix(count + 1, 0);
    for (int k = 0; k < count; ++k) req_prefix[k + 1] = req_prefix[k] + R.ntraj[k];
    if (R.log_x)
        for (uint64_t i = 0; i < req_prefix[count]; ++i) R.log_x[i] = NAN;
    std::vector<Suff> acc(count);
    std::vector<uint64_t> done(count, 0), size(count, 0), still(count, 0);
    std::vector<double> ms_per_traj(count, -1.0);  // launch ms per trajectory, last measured
    std::vector<int32_t> stop(count, -1);
    int round = 0;
    const uint64_t slots = traj_slots(ctx, R.s);
    for (int k = 0; k < count; ++k) {
        if (R.ntraj[k] == 0) stop[k] = PM_STOP_COMPLETE;
        size[k] = R.rse_target > 0 ? std::max<uint64_t>(kMinTrajForTarget, 2 * slots / (uint64_t)count) : R.ntraj[k];
    }
    uint32_t stop_bits = 0;
    double traj_ms = 0;
    std::vector<double> lx;
    for (;;) {
        int running = 0;
        for (int k = 0; k < count; ++k) running += stop[k] < 0;
        if (!running) break;
        Run Q;
        Q.mats = R.mats;
        Q.count = count;
        Q.prepared = dms.data();
        Q.s = R.s;
        Q.seed = R.seed;
        Q.first_traj = R.first_traj;
        Q.model = R.model;
        Q.first_local = done;
        Q.ntraj.assign(count, 0);
        for (int k = 0; k < count; ++k)
            if (stop[k] < 0) Q.ntraj[k] = std::min(size[k], R.ntraj[k] - done[k]);
        if (R.budget_s > 0) {
            const double rem = R.budget_s - elapsed();
            if (rem <= 0) { stop_bits |= ST_TIMEOUT; break; }
            Q.budget_ns = (uint64_t)std::max(1.0, rem * 1e9);
            if (R.rse_target > 0 && round > 0 && count > 1) {  // cheapest to finish first
                double known = 0;
                int nk = 0;
                for (int k = 0; k < count; ++k)
                    if (ms_per_traj[k] > 0) { known += ms_per_traj[k]; ++nk; }
                const double fallback = nk ? known / nk : 1e-3;
                auto price = [&](int k) { return ms_per_traj[k] > 0 ? ms_per_traj[k] : fallback; };
                std::vector<int> cand;
                for (int k = 0; k < count; ++k)
                    if (stop[k] < 0) cand.push_back(k);
                std::stable_sort(cand.begin(), cand.end(), [&](int a, int b) {
                    return (double)still[a] * price(a) < (double)still[b] * price(b);
                });
                const double rem_ms = rem * 1e3;
                double left = (rem_ms > 400.0 ? kRoundShare : 0.95) * rem_ms;
                uint64_t planned = 0;
                for (int k : cand) {
                    uint64_t a = Q.ntraj[k];
                    a = std::min<uint64_t>(a, (uint64_t)std::max(0.0, left / price(k)));
                    if (planned > 0 && a < std::min<uint64_t>(kMinRoundTraj, Q.ntraj[k])) a = 0;
                    Q.ntraj[k] = a;
                    left -= (double)a * price(k);
                    planned += a;
                }
                if (!planned) { stop_bits |= ST_TIMEOUT; break; }  // no room left for a useful launch
                Q.order = cand;
                for (int k = 0; k < count; ++k)
                    if (stop[k] >= 0) Q.order.push_back(k);
            }
        }
        std::vector<pm_result> outs(count);
        Q.outs = outs.data();
        uint64_t tot = 0;
        for (int k = 0; k < count; ++k) tot += Q.ntraj[k];
        if (R.log_x) {
            lx.assign(tot, 0.0);
            Q.log_x = lx.data();
        }
        Staged S;
        st = stage_inputs(ctx, ctx->ws2, Q, S);
        if (st == PM_OK) st = stage_plans(ctx, ctx->ws2, Q, S, nullptr);
        if (st == PM_OK) st = enqueue(ctx, ctx->ws2, Q, S);
        if (st != PM_OK) return st;
        PM_CUDA(cudaStreamSynchronize(ctx->stream));
        st = collect(ctx, ctx->ws2, Q, S, 0.0);
        if (st != PM_OK) return st;
        traj_ms += ctx->last_traj_ms > 0 ? ctx->last_traj_ms : 0;
        h2d += ctx->last_h2d;
        d2h += ctx->last_d2h;
        stop_bits |= S.stop_bits;
        uint64_t off = 0;
        for (int k = 0; k < count; ++k) {
            if (!Q.ntraj[k]) continue;
            outs[k].kernel_ms = 0;  // a launch's time is shared by its matrices: reported once below
            if (outs[k].n_traj > 0 && outs[k].dev_ms > 0) ms_per_traj[k] = outs[k].dev_ms / (double)outs[k].n_traj;
            acc[k].add(outs[k]);
            if (R.log_x)
                std::copy(lx.begin() + off, lx.begin() + off + Q.ntraj[k], R.log_x + req_prefix[k] + done[k]);
            off += Q.ntraj[k];
            done[k] += Q.ntraj[k];  // ids consumed (a stopped launch leaves some unstarted)
            const bool ran_all = outs[k].n_traj == Q.ntraj[k];
            pm_result cur;
            acc[k].fill(cur);
            const bool met = R.rse_target > 0 && cur.n_traj >= std::min(kMinTrajForTarget, R.ntraj[k]) &&
                             cur.n_alive >= 2 && cur.rse <= R.rse_target;
            if (met) {
                stop[k] = PM_STOP_TARGET;
            } else if (!ran_all) {
                stop[k] = (S.stop_bits & ST_CANCELLED) ? PM_STOP_CANCELLED : PM_STOP_TIME;
            } else if (done[k] >= R.ntraj[k]) {
                stop[k] = PM_STOP_COMPLETE;
            } else if (R.rse_target > 0) {  // next round: toward the trajectories the target needs
                const double M = (double)cur.n_traj;
                double need = (cur.rse == cur.rse && cur.n_alive >= 2)
                                  ? 1.1 * M * (cur.rse / R.rse_target) * (cur.rse / R.rse_target)
                                  : 4.0 * M;
                still[k] = (uint64_t)std::max(0.0, need - (double)done[k]);
                need = std::min(need, 5.0 * (double)done[k]);
                size[k] = std::max<uint64_t>(size[k], (uint64_t)std::max(0.0, need - (double)done[k]));
            }
        }
        if (stop_bits) break;
        ++round;
    }
    const double secs = elapsed();
    ctx->last_traj_ms = traj_ms;
    ctx->last_prep_ms = prep_ms;
    ctx->last_h2d = h2d;
    ctx->last_d2h = d2h;
    for (int k = 0; k < count; ++k) {
        pm_result& o = R.outs[k];
        acc[k].fill(o);
        o.kernel_ms = traj_ms;
        o.seconds = secs;
        o.stop = stop[k] >= 0 ? stop[k] : (stop_bits & ST_CANCELLED) ? PM_STOP_CANCELLED : PM_STOP_TIME;
    }
    return stop_status(ctx, stop_bits);
}

}  // namespace


extern "C" {

pm_status pm_context_create(pm_context** out, int device, void* cuda_stream)
{
    if (!out) return PM_EINVAL;
    *out = nullptr;
    pm_context* ctx = new (std::nothrow) pm_context();
    if (!ctx) return PM_ENOMEM;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            ctx->stream = (cudaStream_t)cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            ctx->own_stream = (e == cudaSuccess);
        }
    }
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&ctx->cancel_host, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *(volatile int*)ctx->cancel_host = 0;
        e = cudaHostGetDevicePointer((void**)&ctx->cancel_dev, ctx->cancel_host, 0);
    }
    if (e != cudaSuccess) {
        if (ctx->cancel_host) cudaFreeHost(ctx->cancel_host);
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA;
    }
    *out = ctx;
    return PM_OK;
}

pm_status pm_context_cancel(pm_context* ctx)
{
    if (!ctx || !ctx->cancel_host) return PM_EINVAL;
    __atomic_store_n(ctx->cancel_host, 1, __ATOMIC_SEQ_CST);
    return PM_OK;
}

static void batch_delete(pm_batch* b);

pm_status pm_context_destroy(pm_context* ctx)
{
    if (!ctx) return PM_EINVAL;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (pm_batch* b : ctx->batches) batch_delete(b);
    ctx->batches.clear();
    ctx->ws.release();
    ctx->ws2.release();
    if (ctx->cancel_host) cudaFreeHost(ctx->cancel_host);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return PM_OK;
}

static Sched to_sched(const pm_schedule* s)
{
    Sched o;
    o.vertex_rule = s->vertex_rule; o.initial_dm = s->initial_dm; o.K0 = s->K0; o.K = s->K;
    o.sk = s->sk; o.dm = s->dm; o.precision = s->precision; o.local_cap = s->local_cap; o.theta = s->theta;
    return o;
}

pm_status pm_estimate_batch_ex(pm_context* ctx, const pm_csr* mats, int32_t count, const uint64_t* n_traj,
                               uint64_t first_traj, uint64_t seed, const pm_schedule* schedule, pm_result* outs,
                               double* log_x)
{
    if (!ctx) return PM_EINVAL;
    if (!mats || count < 1 || count > 65535 || !n_traj || !outs) return fail(ctx, PM_EINVAL, "bad batch arguments");
    pm_status st = check_schedule(ctx, schedule);
    if (st != PM_OK) return st;
    for (int k = 0; k < count; ++k) {
        st = check_csr(ctx, &mats[k]);
        if (st != PM_OK) return st;
        if (n_traj[k] >= ((uint64_t)1 << 48)) return fail(ctx, PM_EINVAL, "n_traj above 2^48");
    }
    if (first_traj >= ((uint64_t)1 << 48)) return fail(ctx, PM_EINVAL, "first_traj above 2^48");
    Run R;
    R.mats = mats;
    R.count = count;
    R.ntraj.assign(n_traj, n_traj + count);
    R.first_traj = first_traj;
    R.seed = seed;
    R.s = to_sched(schedule);
    R.outs = outs;
    R.log_x = log_x;
    R.model = schedule->learned ? schedule->learned->img : nullptr;
    R.rse_target = schedule->rse_target;
    R.budget_s = schedule->time_budget_s;
    if (ctx->cancel_host) *(volatile int*)ctx->cancel_host = 0;
    if (R.rse_target > 0 || R.budget_s > 0) return execute_rounds(ctx, R);
    return execute(ctx, R);
}

pm_status estimate_permanent_batch(pm_context* ctx, const pm_csr* mats, int32_t count, const uint64_t* n_traj,
                                   uint64_t seed, const pm_schedule* schedule, pm_result* outs)
{
    return pm_estimate_batch_ex(ctx, mats, count, n_traj, 0, seed, schedule, outs, nullptr);
}

pm_status estimate_permanent(pm_context* ctx, const pm_csr* csr, int32_t n, uint64_t n_traj, uint64_t seed,
                             const pm_schedule* schedule, pm_result* out)
{
    if (!ctx) return PM_EINVAL;
    if (!csr || csr->n != n) return fail(ctx, PM_EINVAL, "n does not match csr->n");
    return pm_estimate_batch_ex(ctx, csr, 1, &n_traj, 0, seed, schedule, out, nullptr);
}

pm_status pm_trace(pm_context* ctx, const pm_csr* csr, uint32_t matrix_index, uint64_t first_traj, uint32_t count,
                   uint64_t seed, const pm_schedule* schedule, int32_t* chosen, int32_t* deg_v, int32_t* dead_step,
                   double* log_x, float* logits, uint32_t logit_stride)
{
    if (!ctx) return PM_EINVAL;
    pm_status st = check_schedule(ctx, schedule);
    if (st != PM_OK) return st;
    st = check_csr(ctx, csr);
    if (st != PM_OK) return st;
    if (count < 1 || matrix_index > 0xFFFF || first_traj + count > ((uint64_t)1 << 48))
        return fail(ctx, PM_EINVAL, "bad trace range");
    if (logits && (logit_stride < 1 || logit_stride > (uint32_t)kMaxDegree + 1))
        return fail(ctx, PM_EINVAL, "logit_stride must be in 1 .. 65535 when logits is given");
    Run R;
    R.mats = csr;
    R.count = 1;
    R.ntraj.assign(1, count);
    R.first_traj = first_traj;
    R.matrix_index0 = matrix_index;
    R.seed = seed;
    R.s = to_sched(schedule);
    R.trace = true;
    R.chosen = chosen;
    R.deg_v = deg_v;
    R.dead_step = dead_step;
    R.log_x = log_x;
    R.logits = logits;
    R.logit_stride = logits ? logit_stride : 0;
    R.model = schedule->learned ? schedule->learned->img : nullptr;
    return execute(ctx, R);
}

pm_status pm_preprocess(pm_context* ctx, const pm_csr* csr, const pm_schedule* schedule, int32_t* ok,
                        uint8_t* keep, double* r, double* c)
{
    if (!ctx) return PM_EINVAL;
    pm_status st = check_schedule(ctx, schedule);
    if (st != PM_OK) return st;
    st = check_csr(ctx, csr);
    if (st != PM_OK) return st;
    Run R;
    R.mats = csr;
    R.count = 1;
    R.ntraj.assign(1, 0);
    R.s = to_sched(schedule);
    R.prep_only = true;
    R.ok_out = ok;
    R.keep_out = keep;
    R.r_out = r;
    R.c_out = c;
    return execute(ctx, R);
}

pm_status pm_philox_blocks(pm_context* ctx, const uint32_t ctr[4], const uint32_t key[2], uint32_t count,
                           uint32_t* out)
{
    if (!ctx || !ctr || !key || !out || count == 0) return PM_EINVAL;
    PM_CUDA(cudaSetDevice(ctx->device));
    pm_status st = grow(ctx, &ctx->ws.arena, &ctx->ws.arena_cap, (size_t)count * 16);
    if (st != PM_OK) return st;
    PM_CUDA(launch_philox(ctr, key, count, (uint32_t*)ctx->ws.arena, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(out, ctx->ws.arena, (size_t)count * 16, cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    return PM_OK;
}

pm_status pm_probe_bandwidth(pm_context* ctx, double* l2_read_gbs, double* smem_read_gbs)
{
    if (!ctx || !l2_read_gbs || !smem_read_gbs) return PM_EINVAL;
    PM_CUDA(cudaSetDevice(ctx->device));
    const size_t bytes = (size_t)64 << 20;  // half of the 126 MB L2
    const int iters = 200;
    DevBuf buf, sink;
    PM_CUDA(cudaMalloc(&buf.p, bytes));
    PM_CUDA(cudaMalloc(&sink.p, 8));
    PM_CUDA(cudaMemsetAsync(buf.p, 1, bytes, ctx->stream));
    PM_CUDA(cudaMemsetAsync(sink.p, 0, 8, ctx->stream));
    cudaEvent_t e0, e1;
    PM_CUDA(cudaEventCreate(&e0));
    PM_CUDA(cudaEventCreate(&e1));
    auto timed = [&](auto&& launch) -> double {
        if (launch() != cudaSuccess) return -1.0;  // warm-up (fills L2)
        cudaEventRecord(e0, ctx->stream);
        if (launch() != cudaSuccess) return -1.0;
        cudaEventRecord(e1, ctx->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    };
    const int grid = ctx->sm_count * 4;
    const double l2_ms = timed([&] {
        return launch_l2_probe(buf.p, bytes, iters, grid, (unsigned long long*)sink.p, ctx->stream);
    });
    const int sm_bytes = 96 << 10, sm_iters = 2000;
    const double sm_ms = timed([&] {
        return launch_smem_probe(sm_bytes, sm_iters, ctx->sm_count * 2, (unsigned long long*)sink.p, ctx->stream);
    });
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    PM_CUDA(cudaGetLastError());
    if (l2_ms <= 0 || sm_ms <= 0) return fail(ctx, PM_ECUDA, "bandwidth probe failed");
    *l2_read_gbs = (double)bytes * iters / (l2_ms * 1e-3) / 1e9;
    *smem_read_gbs = (double)sm_bytes * sm_iters * ctx->sm_count * 2 / (sm_ms * 1e-3) / 1e9;
    return PM_OK;
}

pm_status pm_last_call_info(const pm_context* ctx, pm_call_info* info)
{
    if (!ctx || !info) return PM_EINVAL;
    info->h2d_bytes = ctx->last_h2d;
    info->d2h_bytes = ctx->last_d2h;
    info->traj_kernel_ms = ctx->last_traj_ms;
    info->prep_kernel_ms = ctx->last_prep_ms;
    info->grid = ctx->last_grid;
    info->warps_per_cta = ctx->last_wpc;
    std::memset(&info->first_plan, 0, sizeof(info->first_plan));
    const Plan& p = ctx->last_plan;
    info->first_plan.g = p.g; info->first_plan.groups = p.groups; info->first_plan.staged = p.staged;
    info->first_plan.rc_smem = p.rc_smem; info->first_plan.gstate = p.gstate; info->first_plan.dm_smem = p.dm_smem;
    info->first_plan.pair = p.pair;
    info->first_plan.probe_traj_per_s = info->first_plan.heuristic_traj_per_s = -1.0;
    info->grad_kernel_ms = ctx->last_grad_ms;
    return PM_OK;
}

const char* pm_status_string(pm_status s)
{
    switch (s) {
        case PM_OK: return "PM_OK";
        case PM_EINVAL: return "PM_EINVAL";
        case PM_ENOMEM: return "PM_ENOMEM";
        case PM_ECUDA: return "PM_ECUDA";
        case PM_ETIMEOUT: return "PM_ETIMEOUT";
        case PM_ECANCELLED: return "PM_ECANCELLED";
        case PM_EUNSUPPORTED: return "PM_EUNSUPPORTED";
        case PM_EDEVICE: return "PM_EDEVICE";
    }
    return "PM_UNKNOWN";
}

const char* pm_last_error(const pm_context* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

// ---------------------------------------------------------------------------
// resident batches: device copies, a workspace sized once, an optional CUDA
// graph of the launch sequence and an optional autotuned layout per size class
// ---------------------------------------------------------------------------

}  // extern "C"

struct pm_batch {
    pm_context* ctx = nullptr;
    Workspace ws;
    std::vector<pm_csr> mats;      // device copies owned by the batch
    std::vector<void*> bufs;
    Run R;
    Staged S;
    uint32_t flags = 0;
    // captured segments: preprocessing, trajectories, statistics + read-back
    cudaGraph_t graph[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t exec[3] = {nullptr, nullptr, nullptr};
    cudaGraphNode_t traj_node = nullptr;
    cudaKernelNodeParams traj_params{};
    std::vector<pm_plan_info> info;
    ~pm_batch()
    {
        for (int q = 0; q < 3; ++q) {
            if (exec[q]) cudaGraphExecDestroy(exec[q]);
            if (graph[q]) cudaGraphDestroy(graph[q]);
        }
        for (void* b : bufs) cudaFree(b);
        ws.release();
    }
};

static void batch_delete(pm_batch* b) { delete b; }

namespace {

// Trajectories per second of matrix k under `plan`: a probe launch on up to
// 32 SMs, two trajectories per group, ids far from any run's range.
pm_status probe_plan(pm_context* ctx, pm_batch* b, int k, const Plan& plan, double* rate)
{
    Staged& S = b->S;
    const Run& R = b->R;
    const int count = R.count;
    const int pgrid = std::min(ctx->sm_count, 32);
    const uint32_t per_chunk = (uint32_t)plan.groups * 2;
    const uint64_t ntr = (uint64_t)pgrid * per_chunk;
    const bool scales = R.s.sk != 0, local = R.s.sk == 3, dm = R.s.dm != 0;
    const size_t gstate_bytes = plan.gstate ? global_state_bytes(R.mats[k].n, (int)S.rb, plan.lists != 0) : 0;
    const SlotLayout sl = slot_layout(S.n_max, (int)S.m_max, (int)S.rb, scales, local, dm, gstate_bytes,
                                      R.model != nullptr);
    // probe buffers: plans, chunks, zero prefix, ln X, counters, chunk counter, slots
    Layout L;
    const size_t o_pl = L.take(sizeof(Plan) * count), o_ch = L.take(sizeof(Chunk) * pgrid),
                 o_pf = L.take(8 * (count + 1)), o_lx = L.take(8 * ntr), o_ct = L.take(8 * kCounters * count),
                 o_cc = L.take(8),
                 o_sl = L.take(sl.bytes * (size_t)pgrid * (plan.pair ? pair_cta_warps(R.model != nullptr) : kCtaWarps));
    DevBuf buf;
    PM_CUDA(cudaMalloc(&buf.p, L.off));
    uint8_t* B = (uint8_t*)buf.p;
    std::vector<Plan> plans = S.plans;
    plans[k] = plan;
    std::vector<Chunk> chunks(pgrid);
    for (int c = 0; c < pgrid; ++c) {
        chunks[c].k = k;
        chunks[c].count = per_chunk;
        chunks[c].first = (uint64_t)c * per_chunk;
        chunks[c].slot0 = (uint64_t)c * per_chunk;
    }
    PM_CUDA(cudaMemcpyAsync(B + o_pl, plans.data(), sizeof(Plan) * count, cudaMemcpyHostToDevice, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(B + o_ch, chunks.data(), sizeof(Chunk) * pgrid, cudaMemcpyHostToDevice, ctx->stream));
    PM_CUDA(cudaMemsetAsync(B + o_pf, 0, 8 * (count + 1), ctx->stream));
    PM_CUDA(cudaMemsetAsync(B + o_ct, 0, 8 * kCounters * count, ctx->stream));
    PM_CUDA(cudaMemsetAsync(B + o_cc, 0, 8, ctx->stream));
    TrajParams tp = S.tp;
    tp.plans = (const Plan*)(B + o_pl);
    tp.chunks = (const Chunk*)(B + o_ch);
    tp.n_chunks = pgrid;
    tp.prefix = (const uint64_t*)(B + o_pf);
    tp.first_traj = (uint64_t)1 << 47;
    tp.seed = 0x5eedULL;
    tp.log_x = (double*)(B + o_lx);
    tp.counters = (unsigned long long*)(B + o_ct);
    tp.chunk_counter = (int*)(B + o_cc);
    tp.slots = B + o_sl;
    tp.slot = sl;
    tp.cta_warps = plan.pair ? pair_cta_warps(R.model != nullptr) : kCtaWarps;
    tp.pair_kernel = (plan.pair && R.model == nullptr) ? 1 : 0;
    tp.budget_ns = 0;
    tp.hard_ns = 0;
    tp.cancel = nullptr;
    const int smem = kCtaMiscBytes + learned_smem(R.model != nullptr) + plan.mat_bytes + plan.groups * plan.state_bytes;
    PM_CUDA(cudaEventRecord(b->ws.ev0, ctx->stream));
    PM_CUDA(launch_trajectories(tp, pgrid, smem, false, ctx->stream));
    PM_CUDA(cudaEventRecord(b->ws.ev1, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    float ms = 0;
    PM_CUDA(cudaEventElapsedTime(&ms, b->ws.ev0, b->ws.ev1));
    uint32_t status = 0;
    PM_CUDA(cudaMemcpy(&status, S.tp.status, 4, cudaMemcpyDeviceToHost));
    if (status) return fail(ctx, PM_EDEVICE, "device status " + std::to_string(status) + " in an autotuner probe");
    *rate = ms > 0 ? (double)ntr / (ms * 1e-3) : 0.0;
    return PM_OK;
}

// Layout per matrix: for each size class, time the candidate policies on the
// class's largest matrix and keep the fastest (cached in the context).
pm_status autotune(pm_context* ctx, pm_batch* b, std::vector<Plan>& plans)
{
    Staged& S = b->S;
    const Run& R = b->R;
    const int count = R.count;
    const bool learned = R.model != nullptr;
    const int smem_max = traj_max_smem_bytes();
    // the matrices must be prepared before a probe runs on them
    uint8_t* A = b->ws.arena;
    PM_CUDA(cudaMemsetAsync(A + S.o_status, 0, 4, ctx->stream));
    PM_CUDA(launch_prepare((DevMatrix*)(A + S.o_mats), (const DevInput*)(A + S.o_inputs), count, R.s, S.m_max, S.n_max,
                           (uint32_t*)(A + S.o_status), ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    uint32_t status = 0;
    PM_CUDA(cudaMemcpy(&status, A + S.o_status, 4, cudaMemcpyDeviceToHost));
    if (status & ST_BAD_INPUT) return fail(ctx, PM_EINVAL, "malformed CSR (device validation)");
    if (status) return fail(ctx, PM_EUNSUPPORTED, "device status " + std::to_string(status) + " in preprocessing");
    plans = S.plans;  // heuristic plans from the first stage_plans
    std::map<int, int> rep;  // class -> representative matrix
    for (int k = 0; k < count; ++k) {
        const int c = size_class(R.mats[k].n);
        auto it = rep.find(c);
        if (it == rep.end() || (double)R.mats[k].n * R.mats[k].nnz > (double)R.mats[it->second].n * R.mats[it->second].nnz)
            rep[c] = k;
    }
    for (const auto& cr : rep) {
        const int k = cr.second;
        const int n = R.mats[k].n;
        const int64_t m = R.mats[k].nnz;
        const std::string key = class_key(cr.first, R.s, learned);
        Policy best = policy_of(S.plans[k]);
        double best_rate = -1.0, heur_rate = -1.0;
        auto cached = ctx->tuned.find(key);
        if (cached != ctx->tuned.end()) {
            best = Policy::of_key(cached->second);
        } else {
            const std::vector<Policy> cands = candidate_policies(n, m, (int)S.rb, R.s, smem_max, learned);
            if (cands.size() > 1) {
                for (const Policy& pol : cands) {
                    const Plan pl = plan_for(n, m, (int)S.rb, R.s, smem_max, learned, pol);
                    if (pl.groups < 1) continue;
                    double rate = 0;
                    pm_status st = probe_plan(ctx, b, k, pl, &rate);
                    if (st != PM_OK) return st;
                    if (pol == policy_of(S.plans[k])) heur_rate = rate;
                    if (rate > best_rate) { best_rate = rate; best = pol; }
                }
            }
            ctx->tuned[key] = best.key();
        }
        for (int q = 0; q < count; ++q) {
            if (size_class(R.mats[q].n) != cr.first) continue;
            const Plan pl = plan_for(R.mats[q].n, R.mats[q].nnz, (int)S.rb, R.s, smem_max, learned, best);
            if (pl.groups >= 1) {
                plans[q] = pl;
                b->info[q].tuned = 1;
            }
            b->info[q].probe_traj_per_s = best_rate;
            b->info[q].heuristic_traj_per_s = heur_rate;
        }
    }
    return PM_OK;
}

}  // namespace

extern "C" {

pm_status pm_batch_create(pm_context* ctx, const pm_csr* mats, int32_t count, const uint64_t* n_traj,
                          const pm_schedule* schedule, uint32_t flags, pm_batch** out)
{
    if (!ctx) return PM_EINVAL;
    if (!out || !mats || count < 1 || count > 65535 || !n_traj || (flags & ~3u))
        return fail(ctx, PM_EINVAL, "bad batch arguments");
    *out = nullptr;
    pm_status st = check_schedule(ctx, schedule);
    if (st != PM_OK) return st;
    if (schedule->rse_target != 0) return fail(ctx, PM_EINVAL, "a resident batch runs fixed trajectory counts: rse_target must be 0");
    for (int k = 0; k < count; ++k) {
        st = check_csr(ctx, &mats[k]);
        if (st != PM_OK) return st;
        if (n_traj[k] >= ((uint64_t)1 << 48)) return fail(ctx, PM_EINVAL, "n_traj above 2^48");
    }
    PM_CUDA(cudaSetDevice(ctx->device));
    pm_batch* b = new (std::nothrow) pm_batch();
    if (!b) return PM_ENOMEM;
    b->ctx = ctx;
    b->flags = flags;
    auto bail = [&](pm_status s2) { cudaStreamSynchronize(ctx->stream); delete b; return s2; };
    // device copies of the inputs
    b->mats.resize(count);
    for (int k = 0; k < count; ++k) {
        const pm_csr& c = mats[k];
        const size_t m = (size_t)c.nnz;
        void *rp = nullptr, *ci = nullptr, *va = nullptr;
        cudaError_t e = cudaMalloc(&rp, (c.n + 1) * 8);
        if (e == cudaSuccess) b->bufs.push_back(rp);
        if (e == cudaSuccess) e = cudaMalloc(&ci, std::max<size_t>(m, 1) * 4);
        if (e == cudaSuccess) b->bufs.push_back(ci);
        if (e == cudaSuccess && c.values) e = cudaMalloc(&va, std::max<size_t>(m, 1) * 4);
        if (e == cudaSuccess && va) b->bufs.push_back(va);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rp, c.row_ptr, (c.n + 1) * 8, cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess && m) e = cudaMemcpyAsync(ci, c.col_idx, m * 4, cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess && m && c.values) e = cudaMemcpyAsync(va, c.values, m * 4, cudaMemcpyDefault, ctx->stream);
        if (e != cudaSuccess)
            return bail(fail(ctx, e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA, cudaGetErrorString(e)));
        pm_csr& d = b->mats[k];
        d = c;
        d.on_device = 1;
        d.row_ptr = (const int64_t*)rp;
        d.col_idx = (const int32_t*)ci;
        d.values = (const float*)va;
    }
    Run& R = b->R;
    R.mats = b->mats.data();
    R.count = count;
    R.ntraj.assign(n_traj, n_traj + count);
    R.s = to_sched(schedule);
    R.model = schedule->learned ? schedule->learned->img : nullptr;
    R.budget_ns = (uint64_t)(schedule->time_budget_s * 1e9);
    b->info.assign(count, pm_plan_info{});
    st = stage_inputs(ctx, b->ws, R, b->S, (size_t)ctx->sm_count + count);
    if (st != PM_OK) return bail(st);
    st = stage_plans(ctx, b->ws, R, b->S, nullptr);
    if (st != PM_OK) return bail(st);
    if ((flags & PM_BATCH_AUTOTUNE) && b->S.launch_traj) {
        std::vector<Plan> plans;
        st = autotune(ctx, b, plans);
        if (st != PM_OK) return bail(st);
        st = stage_plans(ctx, b->ws, R, b->S, &plans);
        if (st != PM_OK) return bail(st);
    }
    for (int k = 0; k < count && b->S.launch_traj; ++k) {
        const Plan& p = b->S.plans[k];
        pm_plan_info& I = b->info[k];
        I.g = p.g; I.groups = p.groups; I.staged = p.staged; I.rc_smem = p.rc_smem; I.gstate = p.gstate;
        I.dm_smem = p.dm_smem; I.pair = p.pair;
    }
    if (flags & PM_BATCH_GRAPH) {
        PM_CUDA(cudaStreamSynchronize(ctx->stream));
        for (int seg = 0; seg < 3; ++seg) {
            cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed);
            if (e != cudaSuccess) return bail(fail(ctx, PM_ECUDA, std::string("capture: ") + cudaGetErrorString(e)));
            st = seg == 0 ? enqueue_prep(ctx, b->ws, R, b->S)
                          : seg == 1 ? enqueue_traj(ctx, b->ws, R, b->S) : enqueue_tail(ctx, b->ws, R, b->S);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(ctx->stream, &g);
            b->graph[seg] = g;
            if (st != PM_OK) return bail(st);
            if (e != cudaSuccess) return bail(fail(ctx, PM_ECUDA, std::string("capture: ") + cudaGetErrorString(e)));
            e = cudaGraphInstantiate(&b->exec[seg], b->graph[seg], 0);
            if (e != cudaSuccess)
                return bail(fail(ctx, PM_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e)));
        }
        if (b->S.launch_traj) {
            cudaError_t e;
            size_t nn = 0;
            e = cudaGraphGetNodes(b->graph[1], nullptr, &nn);
            std::vector<cudaGraphNode_t> nodes(nn);
            if (e == cudaSuccess && nn) e = cudaGraphGetNodes(b->graph[1], nodes.data(), &nn);
            const void* fn = traj_kernel_entry(b->S.tp, false);
            for (size_t q = 0; q < nn && e == cudaSuccess; ++q) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nodes[q], &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
                cudaKernelNodeParams kp{};
                if (cudaGraphKernelNodeGetParams(nodes[q], &kp) != cudaSuccess) continue;
                if (kp.func == fn) {
                    b->traj_node = nodes[q];
                    b->traj_params = kp;
                }
            }
            cudaGetLastError();
            if (!b->traj_node) return bail(fail(ctx, PM_ECUDA, "the trajectory kernel node was not found in the graph"));
        }
    }
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    ctx->batches.push_back(b);
    *out = b;
    return PM_OK;
}

pm_status pm_batch_run(pm_batch* b, uint64_t first_traj, uint64_t seed, pm_result* outs, double* log_x)
{
    if (!b) return PM_EINVAL;
    pm_context* ctx = b->ctx;
    if (!outs) return fail(ctx, PM_EINVAL, "outs is NULL");
    if (first_traj >= ((uint64_t)1 << 48)) return fail(ctx, PM_EINVAL, "first_traj above 2^48");
    const auto t0 = std::chrono::steady_clock::now();
    PM_CUDA(cudaSetDevice(ctx->device));
    Run& R = b->R;
    R.first_traj = first_traj;
    R.seed = seed;
    R.outs = outs;
    R.log_x = log_x;
    b->S.tp.first_traj = first_traj;
    b->S.tp.seed = seed;
    if (ctx->cancel_host) *(volatile int*)ctx->cancel_host = 0;
    if (b->exec[0]) {
        if (b->traj_node) {
            void* args[] = {&b->S.tp};
            cudaKernelNodeParams kp = b->traj_params;
            kp.kernelParams = args;
            kp.extra = nullptr;
            PM_CUDA(cudaGraphExecKernelNodeSetParams(b->exec[1], b->traj_node, &kp));
        }
        PM_CUDA(cudaEventRecord(b->ws.ev2, ctx->stream));
        PM_CUDA(cudaGraphLaunch(b->exec[0], ctx->stream));
        PM_CUDA(cudaEventRecord(b->ws.ev0, ctx->stream));
        PM_CUDA(cudaGraphLaunch(b->exec[1], ctx->stream));
        PM_CUDA(cudaEventRecord(b->ws.ev1, ctx->stream));
        PM_CUDA(cudaGraphLaunch(b->exec[2], ctx->stream));
    } else {
        pm_status st = enqueue(ctx, b->ws, R, b->S);
        if (st != PM_OK) return st;
    }
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    b->S.h2d = 0;
    pm_status st = collect(ctx, b->ws, R, b->S, secs);
    R.outs = nullptr;
    R.log_x = nullptr;
    if (st != PM_OK) return st;
    return stop_status(ctx, b->S.stop_bits);
}

pm_status pm_tune_theta(pm_context* ctx, const pm_csr* csr, pm_schedule* schedule, const double* thetas,
                        int32_t count, double probe_s, uint64_t seed, double* scores)
{
    if (!ctx) return PM_EINVAL;
    pm_status st = check_schedule(ctx, schedule);
    if (st != PM_OK) return st;
    st = check_csr(ctx, csr);
    if (st != PM_OK) return st;
    if (!thetas || count < 1 || !(probe_s > 0 && probe_s < INFINITY))
        return fail(ctx, PM_EINVAL, "bad tuning arguments");
    if (schedule->dm != PM_DM_THRS && schedule->dm != PM_DM_TRCK)
        return fail(ctx, PM_EINVAL, "theta tunes the Thrs / Trck DM policies only");
    double best = INFINITY;
    int best_k = -1;
    for (int k = 0; k < count; ++k) {
        if (!(thetas[k] == thetas[k])) return fail(ctx, PM_EINVAL, "theta is NaN");
        pm_schedule s = *schedule;
        s.theta = thetas[k];
        s.rse_target = 0;
        s.time_budget_s = probe_s;
        pm_result r{};
        Run R;
        R.mats = csr;
        R.count = 1;
        R.ntraj.assign(1, (uint64_t)1 << 21);  // the budget ends a probe long before
        R.first_traj = (uint64_t)k << 40;
        R.seed = seed;
        R.s = to_sched(&s);
        R.outs = &r;
        R.model = s.learned ? s.learned->img : nullptr;
        R.budget_s = probe_s;
        st = execute_rounds(ctx, R);
        if (st != PM_OK && st != PM_ETIMEOUT) return st;
        // work-normalised relative variance: RSE^2 x device seconds (lower is better)
        const double score = (r.n_alive >= 2 && r.rse == r.rse && r.dev_ms > 0)
                                 ? r.rse * r.rse * (r.dev_ms * 1e-3) : INFINITY;
        if (scores) scores[k] = score;
        if (score < best) { best = score; best_k = k; }
    }
    if (best_k >= 0) schedule->theta = thetas[best_k];
    ctx->last_error.clear();
    return PM_OK;
}

pm_status pm_layout_set(pm_context* ctx, const pm_schedule* schedule, int32_t n, int64_t nnz,
                        const pm_plan_info* layout)
{
    if (!ctx) return PM_EINVAL;
    pm_status st = check_schedule(ctx, schedule);
    if (st != PM_OK) return st;
    if (!layout || n < 1 || n > kMaxN || nnz < 0) return fail(ctx, PM_EINVAL, "bad layout arguments");
    const Sched s = to_sched(schedule);
    const bool learned = schedule->learned != nullptr;
    Policy pol;
    pol.staged = layout->staged; pol.rc_smem = layout->rc_smem; pol.gstate = layout->gstate;
    pol.g = layout->g; pol.dm_smem = layout->dm_smem; pol.pair = layout->pair;
    const int smem_max = traj_max_smem_bytes();
    const Plan p = plan_for(n, nnz, s.precision == 1 ? 8 : 4, s, smem_max, learned, pol);
    if (p.groups < 1) return fail(ctx, PM_EUNSUPPORTED, "the layout does not fit this size and schedule");
    ctx->tuned[class_key(size_class(n), s, learned)] = pol.key();
    return PM_OK;
}

pm_status pm_batch_plan_info(const pm_batch* b, int32_t k, pm_plan_info* info)
{
    if (!b || !info || k < 0 || k >= (int32_t)b->info.size()) return PM_EINVAL;
    *info = b->info[k];
    return PM_OK;
}

pm_status pm_batch_destroy(pm_batch* b)
{
    if (!b) return PM_EINVAL;
    pm_context* ctx = b->ctx;
    auto it = std::find(ctx->batches.begin(), ctx->batches.end(), b);
    if (it == ctx->batches.end()) return PM_EINVAL;  // not a live batch of its context
    ctx->batches.erase(it);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    delete b;
    return PM_OK;
}

// ---------------------------------------------------------------------------
// serving: a stream of requests, each run in rounds until its RSE target
// ---------------------------------------------------------------------------

}  // extern "C"

namespace {

// one request: its device copy and prepared state (own workspace), and the
// statistics merged over its rounds
struct Request {
    uint64_t id = 0;
    double target_rse = 0, t_submit = 0;
    uint64_t max_traj = 0, done_traj = 0;
    uint32_t rounds = 0;
    pm_csr host{};                // n, nnz (pointers are the device copies)
    std::vector<void*> bufs;
    Workspace ws;                 // arena with the prepared matrix
    DevMatrix dm{};               // prepared descriptor (device pointers into ws)
    size_t bytes = 0;             // device bytes held
    bool prepared = false;
    Suff st;                      // merged statistics of all rounds
    void release()
    {
        for (void* b : bufs) cudaFree(b);
        bufs.clear();
        ws.release();
    }
};

// statistics of a request's merged rounds (seconds, kernel_ms, alg_bytes:
// 0, as documented for pm_request_done)
void fill_result(const Request& q, pm_result& o)
{
    q.st.fill(o);
    o.kernel_ms = o.seconds = 0;
    o.alg_bytes = o.mlp_rows = 0;
}

}  // namespace

struct pm_server {
    pm_context* ctx = nullptr;
    pm_server_cfg cfg{};
    Sched s{};
    const void* model = nullptr;
    std::vector<Request*> queue, active;
    uint64_t next_id = 1, round = 0, bytes_active = 0;
    Workspace ws;  // the rounds' workspace
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
    ~pm_server()
    {
        for (Request* q : queue) { q->release(); delete q; }
        for (Request* q : active) { q->release(); delete q; }
        ws.release();
    }
};

namespace {

// device bytes a request needs: its copy of A plus the prepared state (the
// preprocessing layout of one matrix)
size_t request_bytes(const pm_csr& c, bool fp64)
{
    const size_t n = (size_t)c.n, m = (size_t)c.nnz, rb = fp64 ? 8 : 4;
    const size_t w = c.values ? 1 : 0;
    return (n + 1) * 8 + m * 4 * (1 + w)                          // copy of the input
           + (n + 1) * 4 * 3 + m * (4 * 6 + 1) + m * 4 * 2 * w     // A's int32 CSR/CSC, mask, B0
           + n * rb * 2 + (2 * n + 8) * 2 + (2 * n / 32 + 64) * 4  // scales, degrees, tree
           + (size_t)dm_ws_ints((int)c.n) * 4 + 16 * 256;
}

// copy and prepare (InitialDM, outer SK, degrees, tree) one request
pm_status prepare_request(pm_server* sv, Request* q)
{
    pm_context* ctx = sv->ctx;
    Run R;
    R.mats = &q->host;
    R.count = 1;
    R.ntraj.assign(1, 0);
    R.s = sv->s;
    R.prep_only = true;
    Staged S;
    pm_status st = stage_inputs(ctx, q->ws, R, S);
    if (st != PM_OK) return st;
    S.launch_traj = false;
    st = enqueue(ctx, q->ws, R, S);
    if (st != PM_OK) return st;
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    const uint32_t status = *S.h_status;
    if (status & ST_BAD_INPUT) return fail(ctx, PM_EINVAL, "malformed CSR (device validation)");
    if (status) return fail(ctx, PM_EUNSUPPORTED, "device status " + std::to_string(status) + " in preprocessing");
    q->dm = S.h_mats[0];
    q->prepared = true;
    // the pinned read-back area is not needed any more
    if (q->ws.pinned) { cudaFreeHost(q->ws.pinned); q->ws.pinned = nullptr; q->ws.pinned_cap = 0; }
    return PM_OK;
}

}  // namespace

extern "C" {

pm_status pm_server_create(pm_context* ctx, const pm_server_cfg* cfg, pm_server** out)
{
    if (!ctx) return PM_EINVAL;
    if (!cfg || !out || cfg->traj_min == 0 || cfg->traj_max < cfg->traj_min || cfg->traj_max >= (1u << 24) ||
        cfg->steps_per_round == 0 || cfg->min_traj_done == 0 || cfg->device_budget_bytes == 0)
        return fail(ctx, PM_EINVAL, "bad server configuration");
    pm_status st = check_schedule(ctx, &cfg->schedule);
    if (st != PM_OK) return st;
    if (cfg->schedule.rse_target != 0 || cfg->schedule.time_budget_s != 0)
        return fail(ctx, PM_EINVAL, "server requests carry their own targets: rse_target and time_budget_s must be 0");
    pm_server* sv = new (std::nothrow) pm_server();
    if (!sv) return PM_ENOMEM;
    sv->ctx = ctx;
    sv->cfg = *cfg;
    sv->s = to_sched(&cfg->schedule);
    sv->model = cfg->schedule.learned ? cfg->schedule.learned->img : nullptr;
    *out = sv;
    return PM_OK;
}

pm_status pm_server_submit(pm_server* sv, const pm_csr* csr, double target_rse, uint64_t max_traj, uint64_t* id)
{
    if (!sv) return PM_EINVAL;
    pm_context* ctx = sv->ctx;
    if (!id || !(target_rse > 0) || max_traj == 0) return fail(ctx, PM_EINVAL, "bad request");
    pm_status st = check_csr(ctx, csr);
    if (st != PM_OK) return st;
    PM_CUDA(cudaSetDevice(ctx->device));
    Request* q = new (std::nothrow) Request();
    if (!q) return PM_ENOMEM;
    q->id = sv->next_id++;
    q->target_rse = target_rse;
    q->max_traj = max_traj;
    q->t_submit = sv->now();
    q->bytes = request_bytes(*csr, sv->s.precision == 1);
    // the request keeps its own device copy from now on
    const size_t m = (size_t)csr->nnz;
    void *rp = nullptr, *ci = nullptr, *va = nullptr;
    cudaError_t e = cudaMalloc(&rp, (csr->n + 1) * 8);
    if (e == cudaSuccess) q->bufs.push_back(rp);
    if (e == cudaSuccess) e = cudaMalloc(&ci, std::max<size_t>(m, 1) * 4);
    if (e == cudaSuccess) q->bufs.push_back(ci);
    if (e == cudaSuccess && csr->values) e = cudaMalloc(&va, std::max<size_t>(m, 1) * 4);
    if (e == cudaSuccess && va) q->bufs.push_back(va);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rp, csr->row_ptr, (csr->n + 1) * 8, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess && m) e = cudaMemcpyAsync(ci, csr->col_idx, m * 4, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess && m && va) e = cudaMemcpyAsync(va, csr->values, m * 4, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        q->release();
        delete q;
        return fail(ctx, e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA, cudaGetErrorString(e));
    }
    q->host = *csr;
    q->host.on_device = 1;
    q->host.row_ptr = (const int64_t*)rp;
    q->host.col_idx = (const int32_t*)ci;
    q->host.values = (const float*)va;
    sv->queue.push_back(q);
    *id = q->id;
    return PM_OK;
}

pm_status pm_server_round(pm_server* sv, pm_request_done* done, uint32_t cap, uint32_t* n_done,
                          uint32_t* n_active, uint32_t* n_queued)
{
    if (!sv) return PM_EINVAL;
    pm_context* ctx = sv->ctx;
    if (!done || !n_done || cap == 0) return fail(ctx, PM_EINVAL, "bad round arguments");
    PM_CUDA(cudaSetDevice(ctx->device));
    *n_done = 0;
    auto finish = [&](Request* q, int32_t status) {
        pm_request_done& d = done[(*n_done)++];
        std::memset(&d, 0, sizeof(d));
        d.id = q->id;
        d.status = status;
        fill_result(*q, d.result);
        d.submit_time = q->t_submit;
        d.done_time = sv->now();
        d.rounds = q->rounds;
        q->release();
        delete q;
    };
    // admission: first come first served while the device budget allows; a
    // request larger than the whole budget is refused
    while (!sv->queue.empty() && *n_done < cap) {
        Request* q = sv->queue.front();
        if (q->bytes > sv->cfg.device_budget_bytes) {
            sv->queue.erase(sv->queue.begin());
            finish(q, PM_REQ_REFUSED);
            continue;
        }
        if (sv->bytes_active + q->bytes > sv->cfg.device_budget_bytes && !sv->active.empty()) break;
        sv->queue.erase(sv->queue.begin());
        pm_status st = prepare_request(sv, q);
        if (st != PM_OK) {
            finish(q, PM_REQ_FAILED);
            continue;
        }
        if (!q->dm.ok) {  // no perfect matching: per(A) = 0 exactly
            finish(q, PM_REQ_DONE);
            continue;
        }
        sv->bytes_active += q->bytes;
        sv->active.push_back(q);
    }
    if (!sv->active.empty() && *n_done < cap) {
        // one persistent launch over every active request
        const int count = (int)std::min<size_t>(sv->active.size(), 65535);
        std::vector<pm_csr> dims(count);
        std::vector<DevMatrix> dms(count);
        Run R;
        R.count = count;
        R.ntraj.resize(count);
        // a round lasts about as long as its longest trajectory, so every
        // request gets at least its share of the GPU's trajectory slots
        const uint64_t share = traj_slots(ctx, sv->s) / (uint64_t)count;
        for (int k = 0; k < count; ++k) {
            Request* q = sv->active[k];
            dims[k] = q->host;
            dms[k] = q->dm;
            dms[k].idx = k;
            uint64_t T = sv->cfg.steps_per_round / (uint64_t)std::max(1, q->host.n);
            T = std::max<uint64_t>(T, share);
            T = std::min<uint64_t>(std::max<uint64_t>(T, sv->cfg.traj_min), sv->cfg.traj_max);
            T = std::min<uint64_t>(T, q->max_traj - q->done_traj);
            R.ntraj[k] = std::max<uint64_t>(T, 1);
        }
        R.mats = dims.data();
        R.prepared = dms.data();
        R.first_traj = (sv->round << 24) & (((uint64_t)1 << 48) - 1);
        R.seed = sv->cfg.seed;
        R.s = sv->s;
        R.model = sv->model;
        std::vector<pm_result> outs(count);
        R.outs = outs.data();
        ++sv->round;
        Staged S;
        pm_status st = stage_inputs(ctx, sv->ws, R, S);
        if (st == PM_OK) st = stage_plans(ctx, sv->ws, R, S, nullptr);
        if (st == PM_OK) st = enqueue(ctx, sv->ws, R, S);
        if (st == PM_OK) {
            PM_CUDA(cudaStreamSynchronize(ctx->stream));
            st = collect(ctx, sv->ws, R, S, 0.0);
        }
        if (st != PM_OK) return st;
        std::vector<Request*> keep;
        for (int k = 0; k < count; ++k) {
            Request* q = sv->active[k];
            const pm_result& o = outs[k];
            q->st.add(o);
            q->done_traj += R.ntraj[k];
            q->rounds += 1;
            pm_result cur;
            fill_result(*q, cur);
            const bool met = q->st.n >= sv->cfg.min_traj_done && q->st.alive >= 2 && cur.rse <= q->target_rse;
            const bool spent = q->done_traj >= q->max_traj;
            if ((met || spent) && *n_done < cap) {
                sv->bytes_active -= q->bytes;
                finish(q, met ? PM_REQ_DONE : PM_REQ_BUDGET);
            } else {
                keep.push_back(q);
            }
        }
        for (size_t k = count; k < sv->active.size(); ++k) keep.push_back(sv->active[k]);
        sv->active.swap(keep);
    }
    if (n_active) *n_active = (uint32_t)sv->active.size();
    if (n_queued) *n_queued = (uint32_t)sv->queue.size();
    return PM_OK;
}

double pm_server_clock(const pm_server* sv) { return sv ? sv->now() : 0.0; }

pm_status pm_server_destroy(pm_server* sv)
{
    if (!sv) return PM_EINVAL;
    cudaSetDevice(sv->ctx->device);
    cudaStreamSynchronize(sv->ctx->stream);
    delete sv;
    return PM_OK;
}

// ---------------------------------------------------------------------------
// learned proposal: model, training, parity entry points
// ---------------------------------------------------------------------------

pm_status pm_model_destroy(pm_model* m)
{
    if (!m) return PM_EINVAL;
    cudaSetDevice(m->device);
    cudaFree(m->master);
    cudaFree(m->m1);
    cudaFree(m->m2);
    cudaFree(m->grad);
    cudaFree(m->img);
    delete m;
    return PM_OK;
}

pm_status pm_model_create(pm_context* ctx, const float* params, uint64_t seed, pm_model** out)
{
    if (!ctx || !out) return PM_EINVAL;
    *out = nullptr;
    PM_CUDA(cudaSetDevice(ctx->device));
    const int np = model_param_count();
    std::vector<float> h(np, 0.0f);
    if (params) {
        std::copy(params, params + np, h.begin());
    } else {  // He-style normal initialisation, zero biases
        std::mt19937_64 rng(seed);
        std::normal_distribution<float> nd(0.0f, 1.0f);
        for (int i = 0; i < 64 * 8; ++i) h[i] = nd(rng) * std::sqrt(2.0f / 8.0f);
        for (int i = 0; i < 64 * 64; ++i) h[576 + i] = nd(rng) * std::sqrt(2.0f / 64.0f);
        for (int i = 0; i < 64; ++i) h[4736 + i] = nd(rng) * std::sqrt(1.0f / 64.0f);
    }
    pm_model* m = new (std::nothrow) pm_model();
    if (!m) return PM_ENOMEM;
    m->device = ctx->device;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&m->master, 4 * np);
    if (e == cudaSuccess) e = cudaMalloc(&m->m1, 4 * np);
    if (e == cudaSuccess) e = cudaMalloc(&m->m2, 4 * np);
    if (e == cudaSuccess) e = cudaMalloc(&m->grad, 4 * np);
    if (e == cudaSuccess) e = cudaMalloc(&m->img, model_image_bytes());
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->master, h.data(), 4 * np, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m1, 0, 4 * np, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->m2, 0, 4 * np, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->img, 0, model_image_bytes(), ctx->stream);
    if (e == cudaSuccess) e = launch_model_image(m->master, m->img, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        pm_model_destroy(m);
        return fail(ctx, e == cudaErrorMemoryAllocation ? PM_ENOMEM : PM_ECUDA, cudaGetErrorString(e));
    }
    *out = m;
    return PM_OK;
}

pm_status pm_model_get_params(pm_context* ctx, const pm_model* m, float* params)
{
    if (!ctx || !m || !params) return PM_EINVAL;
    PM_CUDA(cudaSetDevice(ctx->device));
    PM_CUDA(cudaMemcpyAsync(params, m->master, 4 * model_param_count(), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    return PM_OK;
}

pm_status pm_model_set_params(pm_context* ctx, pm_model* m, const float* params)
{
    if (!ctx || !m || !params) return PM_EINVAL;
    PM_CUDA(cudaSetDevice(ctx->device));
    PM_CUDA(cudaMemcpyAsync(m->master, params, 4 * model_param_count(), cudaMemcpyHostToDevice, ctx->stream));
    PM_CUDA(launch_model_image(m->master, m->img, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    return PM_OK;
}

// Model file: 8-byte magic, uint32 version, uint32 parameter count, the FP32
// master parameters (little-endian, the layout of pm_model_get_params), and
// a 64-bit FNV-1a checksum of the parameter bytes.
static const char kModelMagic[8] = {'P', 'M', 'M', 'O', 'D', 'E', 'L', '1'};

static uint64_t fnv1a(const uint8_t* p, size_t n)
{
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ull;
    return h;
}

pm_status pm_model_save(pm_context* ctx, const pm_model* m, const char* path)
{
    if (!ctx || !m || !path) return PM_EINVAL;
    const int np = model_param_count();
    std::vector<float> h(np);
    pm_status st = pm_model_get_params(ctx, m, h.data());
    if (st != PM_OK) return st;
    const uint32_t ver = 1, cnt = (uint32_t)np;
    const uint64_t sum = fnv1a((const uint8_t*)h.data(), 4 * (size_t)np);
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return fail(ctx, PM_EINVAL, std::string("cannot write ") + tmp);
    bool ok = std::fwrite(kModelMagic, 1, 8, f) == 8 && std::fwrite(&ver, 4, 1, f) == 1 &&
              std::fwrite(&cnt, 4, 1, f) == 1 && std::fwrite(h.data(), 4, np, f) == (size_t)np &&
              std::fwrite(&sum, 8, 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return fail(ctx, PM_EINVAL, std::string("cannot write ") + path);
    }
    return PM_OK;
}

pm_status pm_model_load(pm_context* ctx, const char* path, pm_model** out)
{
    if (!ctx || !path || !out) return PM_EINVAL;
    *out = nullptr;
    const int np = model_param_count();
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(ctx, PM_EINVAL, std::string("cannot read ") + path);
    char magic[8];
    uint32_t ver = 0, cnt = 0;
    uint64_t sum = 0;
    std::vector<float> h(np);
    char extra;
    const bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kModelMagic, 8) == 0 &&
                    std::fread(&ver, 4, 1, f) == 1 && ver == 1 && std::fread(&cnt, 4, 1, f) == 1 &&
                    cnt == (uint32_t)np && std::fread(h.data(), 4, np, f) == (size_t)np &&
                    std::fread(&sum, 8, 1, f) == 1 && std::fread(&extra, 1, 1, f) == 0 &&
                    sum == fnv1a((const uint8_t*)h.data(), 4 * (size_t)np);
    std::fclose(f);
    if (!ok) return fail(ctx, PM_EINVAL, std::string("not a model file of this library: ") + path);
    return pm_model_create(ctx, h.data(), 0, out);
}

pm_status pm_merge_results(const pm_result* parts, int32_t count, pm_result* out)
{
    if (!parts || count < 1 || !out) return PM_EINVAL;
    Suff s;
    for (int32_t i = 0; i < count; ++i) s.add(parts[i]);
    s.fill(*out);
    out->stop = PM_STOP_COMPLETE;
    for (int32_t i = 0; i < count; ++i) out->stop = std::max(out->stop, parts[i].stop);
    return PM_OK;
}

// small device buffers for the parity entry points (freed on return)
pm_status pm_mlp_forward(pm_context* ctx, const pm_model* m, const float* X, uint64_t B, float* out)
{
    if (!ctx || !m || !X || !out || B == 0 || B > (1ull << 30)) return PM_EINVAL;
    PM_CUDA(cudaSetDevice(ctx->device));
    DevBuf bx, bo;
    PM_CUDA(cudaMalloc(&bx.p, 32 * B));
    PM_CUDA(cudaMalloc(&bo.p, 4 * B));
    PM_CUDA(cudaMemcpyAsync(bx.p, X, 32 * B, cudaMemcpyHostToDevice, ctx->stream));
    PM_CUDA(launch_mlp_forward(m->img, (const float*)bx.p, (int)B, (float*)bo.p, ctx->sm_count, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(out, bo.p, 4 * B, cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    return PM_OK;
}

// group codes (index within the group << 16 | group size) that tile rows
// [0, B) with consecutive, complete groups
static bool groups_valid(const uint32_t* g, uint64_t B)
{
    uint64_t r = 0;
    while (r < B) {
        const uint32_t size = g[r] & 0xFFFFu;
        if ((g[r] >> 16) != 0 || size == 0 || r + size > B) return false;
        for (uint32_t k = 0; k < size; ++k)
            if (g[r + k] != ((k << 16) | size)) return false;
        r += size;
    }
    return true;
}

pm_status pm_mlp_gradient(pm_context* ctx, const pm_model* m, const float* X, const float* T, const uint32_t* group,
                          uint64_t B, float* grad, double* loss)
{
    if (!ctx || !m || !X || !T || !grad || B == 0 || B > (1ull << 30)) return PM_EINVAL;
    if (group && !groups_valid(group, B)) return fail(ctx, PM_EINVAL, "group codes do not tile the rows");
    PM_CUDA(cudaSetDevice(ctx->device));
    DevBuf bx, bt, bp, bl, bg, br;
    PM_CUDA(cudaMalloc(&bx.p, 32 * B));
    PM_CUDA(cudaMalloc(&bt.p, 4 * B));
    PM_CUDA(cudaMalloc(&bp.p, 4 * B));
    PM_CUDA(cudaMalloc(&bl.p, 8));
    if (group) {
        PM_CUDA(cudaMalloc(&bg.p, 4 * B));
        PM_CUDA(cudaMalloc(&br.p, 4 * B));
        PM_CUDA(cudaMemcpyAsync(bg.p, group, 4 * B, cudaMemcpyHostToDevice, ctx->stream));
    }
    std::vector<int> perm(B);
    for (uint64_t i = 0; i < B; ++i) perm[i] = (int)i;
    PM_CUDA(cudaMemcpyAsync(bx.p, X, 32 * B, cudaMemcpyHostToDevice, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(bt.p, T, 4 * B, cudaMemcpyHostToDevice, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(bp.p, perm.data(), 4 * B, cudaMemcpyHostToDevice, ctx->stream));
    PM_CUDA(cudaMemsetAsync(m->grad, 0, 4 * model_param_count(), ctx->stream));
    PM_CUDA(cudaMemsetAsync(bl.p, 0, 8, ctx->stream));
    DevBuf bw;
    PM_CUDA(cudaMalloc(&bw.p, mlp_grad_workspace_bytes(ctx->sm_count)));
    PM_CUDA(cudaMemsetAsync(bw.p, 0, 4, ctx->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PM_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(ctx, PM_ECUDA, "cudaEventCreate");
    }
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } evg{e0, e1};
    PM_CUDA(cudaEventRecord(e0, ctx->stream));
    PM_CUDA(launch_mlp_grad(m->img, (const float*)bx.p, (const float*)bt.p, (const int*)bp.p, 0, (int)B,
                            (const uint32_t*)bg.p, (float*)br.p, m->grad, (double*)bl.p, ctx->sm_count, bw.p,
                            ctx->stream));
    PM_CUDA(cudaEventRecord(e1, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(grad, m->grad, 4 * model_param_count(), cudaMemcpyDeviceToHost, ctx->stream));
    double l = 0;
    int werr = 0;
    PM_CUDA(cudaMemcpyAsync(&l, bl.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(&werr, bw.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (werr) return fail(ctx, PM_EDEVICE, "a tensor-core completion wait ran out in the gradient kernel");
    float gms = 0.f;
    ctx->last_grad_ms = cudaEventElapsedTime(&gms, e0, e1) == cudaSuccess ? gms : -1.0;
    if (loss) *loss = l;
    return PM_OK;
}

// record pairs of one or more matrices into device buffers (trajectory kernel in record mode)
static pm_status record_into(pm_context* ctx, const pm_csr* mats, int32_t count, const uint64_t* ntraj,
                             uint64_t first, uint32_t matrix_index0, uint64_t seed, const pm_schedule* teacher,
                             float* dfeat, float* dtarget, unsigned long long* dkey, uint32_t* dgroup,
                             unsigned long long* dcount, unsigned long long cap)
{
    Run R;
    R.mats = mats;
    R.count = count;
    R.ntraj.assign(ntraj, ntraj + count);
    R.first_traj = first;
    R.matrix_index0 = matrix_index0;
    R.seed = seed;
    R.s = to_sched(teacher);
    R.rec_feat = dfeat;
    R.rec_target = dtarget;
    R.rec_key = dkey;
    R.rec_group = dgroup;
    R.rec_count = dcount;
    R.rec_cap = cap;
    std::vector<pm_result> outs(count);
    R.outs = outs.data();
    return execute(ctx, R);
}

static pm_status check_teacher(pm_context* ctx, const pm_schedule* t)
{
    pm_status st = check_schedule(ctx, t);
    if (st != PM_OK) return st;
    if (t->learned || t->precision != 0 || (t->sk != 1 && t->sk != 2))
        return fail(ctx, PM_EINVAL, "the teacher must be an FP32 Fixed/Adaptive SK schedule");
    return PM_OK;
}

pm_status pm_record_pairs(pm_context* ctx, const pm_csr* csr, uint32_t matrix_index, uint64_t first_traj, uint32_t count,
                          uint64_t seed, const pm_schedule* teacher, uint64_t cap, float* feat, float* target,
                          uint64_t* key, uint32_t* group, uint64_t* n_out)
{
    if (!ctx || !csr || !feat || !target || !key || !n_out || cap == 0 || count == 0 || matrix_index > 0xFFFF)
        return PM_EINVAL;
    pm_status st = check_teacher(ctx, teacher);
    if (st != PM_OK) return st;
    st = check_csr(ctx, csr);
    if (st != PM_OK) return st;
    PM_CUDA(cudaSetDevice(ctx->device));
    DevBuf bf, bt, bk, bg, bc;
    PM_CUDA(cudaMalloc(&bf.p, 32 * cap));
    PM_CUDA(cudaMalloc(&bt.p, 4 * cap));
    PM_CUDA(cudaMalloc(&bk.p, 8 * cap));
    PM_CUDA(cudaMalloc(&bg.p, 4 * cap));
    PM_CUDA(cudaMalloc(&bc.p, 16));
    PM_CUDA(cudaMemsetAsync(bc.p, 0, 16, ctx->stream));
    const uint64_t nt = count;
    st = record_into(ctx, csr, 1, &nt, first_traj, matrix_index, seed, teacher, (float*)bf.p, (float*)bt.p,
                     (unsigned long long*)bk.p, (uint32_t*)bg.p, (unsigned long long*)bc.p, cap);
    if (st != PM_OK) return st;
    unsigned long long c[2] = {0, 0};
    PM_CUDA(cudaMemcpy(c, bc.p, 16, cudaMemcpyDeviceToHost));
    const uint64_t kept = std::min<uint64_t>(c[1], cap);  // the filled prefix
    PM_CUDA(cudaMemcpy(feat, bf.p, 32 * kept, cudaMemcpyDeviceToHost));
    PM_CUDA(cudaMemcpy(target, bt.p, 4 * kept, cudaMemcpyDeviceToHost));
    PM_CUDA(cudaMemcpy(key, bk.p, 8 * kept, cudaMemcpyDeviceToHost));
    if (group) PM_CUDA(cudaMemcpy(group, bg.p, 4 * kept, cudaMemcpyDeviceToHost));
    *n_out = kept;
    return PM_OK;
}

pm_status pm_model_train(pm_context* ctx, pm_model* m, const pm_csr* mats, int32_t count, const pm_train_cfg* cfg,
                         pm_train_report* report)
{
    if (!ctx || !m || !mats || count < 1 || count > 65535 || !cfg || cfg->n_pairs == 0 || cfg->epochs < 1 ||
        cfg->batch < 16 || cfg->n_pairs > (1ull << 31) || (cfg->objective != PM_OBJ_MSE && cfg->objective != PM_OBJ_CENTRED) ||
        cfg->reserved != 0)
        return fail(ctx, PM_EINVAL, "bad training arguments");
    pm_status st = check_teacher(ctx, &cfg->teacher);
    if (st != PM_OK) return st;
    for (int k = 0; k < count; ++k) {
        st = check_csr(ctx, &mats[k]);
        if (st != PM_OK) return st;
    }
    PM_CUDA(cudaSetDevice(ctx->device));
    const auto t0 = std::chrono::steady_clock::now();
    const uint64_t want = cfg->n_pairs;
    const bool centred = cfg->objective == PM_OBJ_CENTRED;
    // one recording run sized to give about 1.5 x `want` pairs (about 2 per
    // step), into a buffer that cannot overflow (a trajectory records each
    // edge at most once): the recorded set does not depend on the order in
    // which the device's warps finish
    std::vector<uint64_t> nt(count);
    uint64_t cap = 1;
    for (int k = 0; k < count; ++k) {
        const uint64_t per_traj = 2ull * (uint64_t)mats[k].n;
        const uint64_t goal = want + want / 2;
        nt[k] = std::max<uint64_t>(1, (goal + (uint64_t)count * per_traj - 1) / ((uint64_t)count * per_traj));
        cap += nt[k] * (uint64_t)std::max<int64_t>(1, mats[k].nnz);
    }
    cap = std::min<uint64_t>(std::min<uint64_t>(cap, 16 * want + 1024), (1ull << 31) - 1);
    DevBuf bf, bt, bk, bg, bc, bp, bl, br;
    PM_CUDA(cudaMalloc(&bf.p, 32 * cap));
    PM_CUDA(cudaMalloc(&bt.p, 4 * cap));
    PM_CUDA(cudaMalloc(&bk.p, 8 * cap));
    PM_CUDA(cudaMalloc(&bg.p, 4 * cap));
    PM_CUDA(cudaMalloc(&bc.p, 16));
    PM_CUDA(cudaMemsetAsync(bc.p, 0, 16, ctx->stream));
    st = record_into(ctx, mats, count, nt.data(), 0, 0, cfg->seed, &cfg->teacher, (float*)bf.p, (float*)bt.p,
                     (unsigned long long*)bk.p, (uint32_t*)bg.p, (unsigned long long*)bc.p, cap);
    if (st != PM_OK) return st;
    unsigned long long cnt[2] = {0, 0};
    PM_CUDA(cudaMemcpy(cnt, bc.p, 16, cudaMemcpyDeviceToHost));
    const uint64_t N_all = std::min<uint64_t>(cnt[1], cap);  // the filled prefix: whole steps only
    const auto t1 = std::chrono::steady_clock::now();
    if (N_all < 16) return fail(ctx, PM_EINVAL, "the teacher produced too few pairs");
    // the steps in a fixed order (key, then content: keys repeat across
    // matrices), whole steps up to `want` pairs
    std::vector<uint32_t> gc(N_all);
    std::vector<unsigned long long> keys(N_all);
    std::vector<float> fh(8 * N_all), tg(N_all);
    PM_CUDA(cudaMemcpy(gc.data(), bg.p, 4 * N_all, cudaMemcpyDeviceToHost));
    PM_CUDA(cudaMemcpy(keys.data(), bk.p, 8 * N_all, cudaMemcpyDeviceToHost));
    PM_CUDA(cudaMemcpy(fh.data(), bf.p, 32 * N_all, cudaMemcpyDeviceToHost));
    PM_CUDA(cudaMemcpy(tg.data(), bt.p, 4 * N_all, cudaMemcpyDeviceToHost));
    std::vector<uint64_t> starts;
    for (uint64_t i = 0; i < N_all;) {
        const uint32_t size = gc[i] & 0xFFFFu;
        if ((gc[i] >> 16) != 0 || size == 0 || i + size > N_all) return fail(ctx, PM_EDEVICE, "recorded groups are torn");
        starts.push_back(i);
        i += size;
    }
    std::sort(starts.begin(), starts.end(), [&](uint64_t x, uint64_t y) {
        if (keys[x] != keys[y]) return keys[x] < keys[y];
        const uint32_t sx = gc[x] & 0xFFFFu, sy = gc[y] & 0xFFFFu;
        if (sx != sy) return sx < sy;
        const int c = std::memcmp(&fh[8 * x], &fh[8 * y], 32 * (size_t)sx);
        if (c != 0) return c < 0;
        return std::memcmp(&tg[x], &tg[y], 4 * (size_t)sx) < 0;
    });
    std::vector<uint64_t> kept;
    uint64_t N = 0;
    for (uint64_t s0 : starts) {
        const uint32_t size = gc[s0] & 0xFFFFu;
        if (N + size > want) break;
        kept.push_back(s0);
        N += size;
    }
    if (N < 16) return fail(ctx, PM_EINVAL, "the teacher produced too few pairs");
    // start the output bias at the mean target
    double mean = 0;
    for (uint64_t s0 : kept)
        for (uint32_t q = 0; q < (gc[s0] & 0xFFFFu); ++q) mean += tg[s0 + q];
    mean /= (double)N;
    if (m->step == 0) {
        const float b3 = (float)mean;
        PM_CUDA(cudaMemcpy(m->master + 4800, &b3, 4, cudaMemcpyHostToDevice));
        PM_CUDA(launch_model_image(m->master, m->img, ctx->stream));
    }
    // shuffled order and batches: single pairs for the squared error; whole
    // steps (kept consecutive, batches cut between steps) for the centred loss
    std::mt19937_64 rng(cfg->seed ^ 0x9E3779B97F4A7C15ull);
    std::vector<int> perm;
    std::vector<uint64_t> cuts;  // batch b = perm[cuts[b] .. cuts[b + 1])
    perm.reserve(N);
    if (centred) {
        std::shuffle(kept.begin(), kept.end(), rng);
        cuts.push_back(0);
        for (uint64_t s0 : kept) {
            const uint32_t size = gc[s0] & 0xFFFFu;
            if (perm.size() - cuts.back() + size > (uint64_t)cfg->batch && perm.size() > cuts.back())
                cuts.push_back(perm.size());
            for (uint32_t k = 0; k < size; ++k) perm.push_back((int)(s0 + k));
        }
        cuts.push_back(perm.size());
    } else {
        for (uint64_t s0 : kept)
            for (uint32_t k = 0; k < (gc[s0] & 0xFFFFu); ++k) perm.push_back((int)(s0 + k));
        std::shuffle(perm.begin(), perm.end(), rng);
        for (uint64_t r = 0; r < N; r += (uint64_t)cfg->batch) cuts.push_back(r);
        cuts.push_back(N);
    }
    uint64_t max_batch = 0;
    for (size_t b = 0; b + 1 < cuts.size(); ++b) max_batch = std::max<uint64_t>(max_batch, cuts[b + 1] - cuts[b]);
    PM_CUDA(cudaMalloc(&bp.p, 4 * N));
    PM_CUDA(cudaMemcpy(bp.p, perm.data(), 4 * N, cudaMemcpyHostToDevice));
    if (centred) PM_CUDA(cudaMalloc(&br.p, 4 * max_batch));
    DevBuf bw;  // error word and partial sums of the gradient reduction
    PM_CUDA(cudaMalloc(&bw.p, mlp_grad_workspace_bytes(ctx->sm_count)));
    PM_CUDA(cudaMemsetAsync(bw.p, 0, 4, ctx->stream));
    const uint64_t steps_per_epoch = cuts.size() - 1;
    const uint64_t total_steps = steps_per_epoch * (uint64_t)cfg->epochs;
    PM_CUDA(cudaMalloc(&bl.p, 8 * total_steps));
    PM_CUDA(cudaMemsetAsync(bl.p, 0, 8 * total_steps, ctx->stream));
    uint64_t sidx = 0;
    NvtxScope nv("pm train");
    for (int ep = 0; ep < cfg->epochs; ++ep) {
        for (uint64_t b = 0; b < steps_per_epoch; ++b, ++sidx) {
            const uint64_t row0 = cuts[b];
            const int B = (int)(cuts[b + 1] - cuts[b]);
            PM_CUDA(cudaMemsetAsync(m->grad, 0, 4 * model_param_count(), ctx->stream));
            PM_CUDA(launch_mlp_grad(m->img, (const float*)bf.p, (const float*)bt.p, (const int*)bp.p, (int64_t)row0, B,
                                    centred ? (const uint32_t*)bg.p : nullptr, (float*)br.p, m->grad,
                                    (double*)bl.p + sidx, ctx->sm_count, bw.p, ctx->stream));
            ++m->step;
            PM_CUDA(launch_adam(m->master, m->m1, m->m2, m->grad, cfg->lr, cfg->beta1, cfg->beta2, cfg->eps, m->step,
                                m->img, ctx->stream));
        }
    }
    std::vector<double> losses(total_steps);
    int werr = 0;
    PM_CUDA(cudaMemcpyAsync(losses.data(), bl.p, 8 * total_steps, cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaMemcpyAsync(&werr, bw.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (werr) return fail(ctx, PM_EDEVICE, "a tensor-core completion wait ran out in the gradient kernel");
    const auto t2 = std::chrono::steady_clock::now();
    if (report) {
        std::memset(report, 0, sizeof(*report));
        report->loss_first = losses.front();
        double s = 0;
        for (uint64_t q = total_steps - steps_per_epoch; q < total_steps; ++q) s += losses[q];
        report->loss_last = s / (double)steps_per_epoch;
        report->n_pairs = N;
        report->steps = (int32_t)total_steps;
        report->seconds_record = std::chrono::duration<double>(t1 - t0).count();
        report->seconds_train = std::chrono::duration<double>(t2 - t1).count();
    }
    return PM_OK;
}

}  // extern "C"
