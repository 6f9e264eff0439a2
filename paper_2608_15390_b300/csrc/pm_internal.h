// pm_internal.h -- structures shared by the library's kernels and its host
// code (not part of the C ABI).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pm {

constexpr int kWarp = 32;
// largest order accepted; live degrees are uint16 (0xFFFF marks an inactive
// vertex), so a matrix whose rows or columns hold more than kMaxDegree
// entries is rejected as unsupported
constexpr int kMaxN = 1 << 22;
constexpr int kMaxDegree = 65534;
constexpr int kMaxTreeLevels = 4;
constexpr int kMaxRngAttempts = 256;
// Philox draw index of a step's sampling word for the bounded-work Local
// repair (beyond every draw the partner sampling can take)
constexpr uint32_t kLocalDraw = 2048;

// device status word bits
enum : uint32_t {
    ST_RNG_EXHAUSTED = 1u << 0,
    ST_BAD_INPUT = 1u << 1,
    ST_INTERNAL = 1u << 2,
    ST_CAPACITY = 1u << 3,
    // not errors: the launch stopped starting trajectories early (every
    // trajectory it started ran to its end; the others keep ln X = NaN)
    ST_TIMEOUT = 1u << 4,     // the launch's time budget ran out
    ST_CANCELLED = 1u << 5,   // the context's cancel flag was raised
};
constexpr uint32_t kStatusStopBits = ST_TIMEOUT | ST_CANCELLED;

// Original input matrix A on the device (int32 offsets, validated).
struct DevInput {
    int n, m;
    const int64_t* rp64;    // caller's row pointer
    const int32_t* ci_in;   // caller's column indices
    const float* val_in;    // caller's values or nullptr
};

// A prepared matrix: B0 = A after the initial DM, its CSC view, the outer
// scaling and the initial minimum-degree state.  Everything a trajectory
// reads; lives in the context's arena.
struct DevMatrix {
    int n, m;            // order, nnz of B0
    int ok;              // initial DM found a perfect matching
    int unit_scale;      // binary and r0 = c0 = 1: every proposal is uniform
    int idx;             // matrix index in the Philox counter
    int matched;         // dm_ws starts with a perfect matching of B0 (mr[n], mc[n]) from the initial DM
    // A (validated copy with int32 offsets) and its CSC view
    int* a_rp; int* a_ci; float* a_val; int* a_cp; int* a_ri; int* a_ce;
    uint8_t* keep;       // [m_A] edge survives the initial DM
    int m_a;
    int pad2;
    // B0
    int* rp; int* ci; float* rv;          // CSR
    int* cp; int* ri; float* cv; int* ce; // CSC; ce = CSR edge id of a CSC entry
    void* r0; void* c0;                   // outer scaling (float or double)
    uint16_t* deg0;                       // [2n] initial live degrees
    uint32_t* tree0;                      // initial min-degree tree levels
    int* dm_ws;                           // [dm_ws_ints] initial-DM workspace
};

struct Sched {
    int vertex_rule, initial_dm, K0, K, sk, dm, precision;
    int local_cap;  // 0: the Local repair of Eq. 5; L > 0: its bounded-work variant
    double theta;
};

// min-degree tree geometry for 2n leaves: level l (1..nlev) holds the
// minimum packed key of 32 entries of level l-1 (level 0 = leaves).
struct TreeGeom {
    int n2, nlev, idb;
    uint32_t dcap;
    int off[kMaxTreeLevels + 1];
    int size[kMaxTreeLevels + 1];
    int total;           // words of levels 1..nlev
};

__host__ __device__ inline TreeGeom tree_geom(int n)
{
    TreeGeom g{};
    g.n2 = 2 * n;
    int idb = 0;
    while ((1 << idb) < g.n2) ++idb;
    g.idb = idb < 1 ? 1 : idb;
    g.dcap = (1u << (32 - g.idb)) - 2u;
    int sz = g.n2, off = 0, l = 0;
    g.size[0] = sz;
    while (sz > kWarp && l < kMaxTreeLevels) {
        sz = (sz + kWarp - 1) / kWarp;
        ++l;
        g.off[l] = off;
        g.size[l] = sz;
        off += sz;
    }
    g.nlev = l;
    g.total = off;
    return g;
}

// per-warp global scratch layout for one trajectory slot
struct SlotLayout {
    size_t state;         // global-state plans: degrees, tree, r, c, lists
    size_t r, c;          // Real[n_max] each
    size_t stamp;         // int[n_max]
    size_t tmp_id;        // int[n_max]
    size_t tmp_val;       // Real[n_max]
    size_t list_r, list_c;// int[n_max] each
    size_t mask;          // uint8[m_max]
    size_t dm;            // int[dm ints]
    size_t logit;         // float[2][n_max] logits of long candidate lists (learned proposal)
    size_t bytes;
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline int dm_ws_ints(int n) { return 21 * n + 8; }

// shared bytes of the initial DM with A's adjacency staged beside its
// workspace: int32 row/column pointers, uint16 column/row indices
__host__ __device__ inline size_t prep_stage_bytes(int n, int64_t m)
{
    const size_t a = 16;
    auto up = [a](size_t x) { return (x + a - 1) / a * a; };
    return up((size_t)dm_ws_ints(n) * 4) + 2 * up((size_t)(n + 1) * 4) + 2 * up((size_t)m * 2);
}

inline int group_state_bytes(int n, int64_t m, int real_bytes, bool rc_smem, bool lists, bool learned,
                             bool dm_smem);

inline SlotLayout slot_layout(int n_max, int m_max, int real_bytes, bool scales, bool local, bool dm,
                              size_t gstate_bytes, bool learned)
{
    SlotLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t p = o; o = align_up(o + bytes, 256); return p; };
    L.state = gstate_bytes ? take(gstate_bytes) : 0;
    L.r = scales ? take((size_t)n_max * real_bytes) : 0;
    L.c = scales ? take((size_t)n_max * real_bytes) : 0;
    L.stamp = local ? take((size_t)n_max * 4) : 0;
    L.tmp_id = local ? take((size_t)n_max * 4) : 0;
    L.tmp_val = local ? take((size_t)n_max * real_bytes) : 0;
    L.list_r = local ? take((size_t)n_max * 4) : 0;
    L.list_c = local ? take((size_t)n_max * 4) : 0;
    L.mask = dm ? take((size_t)m_max) : 0;
    L.dm = dm ? take((size_t)dm_ws_ints(n_max) * 4) : 0;
    L.logit = learned ? take((size_t)n_max * 8) : 0;  // two lists: one per half-warp trajectory of a pair plan
    L.bytes = align_up(o, 256);
    if (L.bytes == 0) L.bytes = 256;
    return L;
}

// Execution plan of one matrix, chosen on the host: a trajectory is run by a
// group of g warps (the leader warp does the sequential step, the whole group
// the SK sweeps); `groups` groups share a CTA; the CTA optionally stages the
// matrix indices (uint16) in shared memory; the scaling vectors live in
// shared memory (rc_smem) or in the group's global slot.
struct Plan {
    int g, groups, staged, rc_smem, lists;
    int gstate;        // trajectory state in the group's global slot (large n)
    int dm_smem;       // the inner DM's workspace and edge mask in shared memory
    int state_bytes;   // shared bytes of one group (pair plans: of one trajectory)
    int mat_bytes;     // shared bytes of the staged matrix (0 if not staged)
    int pair;          // two trajectories per warp, one per 16-lane half (`groups`
                       // trajectory states, even, on groups / 2 warps)
};

// shared bytes of one trajectory of a pair plan: degrees, tree and (learned
// proposal) a 16-row feature tile
inline int pair_state_bytes(int n, bool learned)
{
    const TreeGeom G = tree_geom(n);
    size_t b = align_up((size_t)((2 * n + 7) & ~7) * 2, 16) + align_up((size_t)G.total * 4, 16);
    if (learned) b += 16 * 24 * 2;
    return (int)b;
}

// a run of trajectories first .. first + count - 1 (indices inside matrix k);
// trajectory first + q writes its ln X to log_x[slot0 + q]
struct Chunk {
    int k;
    uint32_t count;
    uint64_t first;
    uint64_t slot0;
};

// per-matrix counters of a launch: DM calls, full SK iterations, Local
// repairs, algorithmic bytes, network rows, trajectory nanoseconds
constexpr int kCounters = 6;
constexpr int kCtaWarps = 16;            // 512 threads, one CTA per SM
// The pair-only kernel of the scaled and uniform proposals (every plan of
// the launch a pair plan): 24 warps, as their pair path fits in 80 registers
// a thread.  The learned proposal's pair path runs in the general kernel
// (16 warps of 128 registers): with fewer registers its two-tile network
// spills, which cost more than the extra warps gained (they help only where
// shared memory holds more than 32 trajectory states).
constexpr int kPairCtaWarps = 24;
__host__ __device__ constexpr int pair_cta_warps(bool learned) { return learned ? kCtaWarps : kPairCtaWarps; }
constexpr int kCtaMiscBytes = 64;
constexpr int kGroupMiscInts = 32;

struct TrajParams {
    const DevMatrix* mats;
    const Plan* plans;        // [count]
    const Chunk* chunks;      // [n_chunks]
    int n_chunks;
    int count;
    int n_max;
    const uint64_t* prefix;   // [count + 1] exclusive prefix of trajectories per matrix
    uint64_t first_traj;
    uint64_t seed;
    Sched s;
    double* log_x;            // [prefix[count]]
    unsigned long long* counters;  // [count][kCounters], see kCounters
    int* chunk_counter;
    uint32_t* status;
    uint8_t* slots;           // per-group global scratch, cta_warps slots per CTA
    int cta_warps;            // warps of a CTA: kCtaWarps, or kPairCtaWarps for the pair-only kernel
    int pair_kernel;          // launch the pair-only kernel (scaled / uniform proposal, every plan a pair plan)
    SlotLayout slot;
    // trace outputs (nullptr when not tracing)
    int32_t* chosen;
    int32_t* deg_v;
    int32_t* dead_step;
    float* trace_logits;      // [T][n][logit_stride] logits of the live candidates (learned proposal)
    int logit_stride;         // candidates kept per step in trace_logits
    // run control: no trajectory starts once budget_ns (> 0) nanoseconds of
    // device time (%globaltimer) have passed since the launch's first CTA
    // began (t_start, zeroed before the launch), or once *cancel != 0
    // (host-mapped flag, may be nullptr); started trajectories run to the end
    uint64_t budget_ns;
    unsigned long long* t_start;
    const volatile int* cancel;
    // hard limit (0: none): a trajectory still running hard_ns after the
    // launch's start is abandoned and left out of the sample (ln X = NaN),
    // so no single long trajectory can hold the launch far past its budget
    uint64_t hard_ns;
    // learned proposal: BF16 device image of the network, or nullptr
    const void* model;
    // recording of (features, SK target) pairs, or rec_feat == nullptr
    float* rec_feat;          // [cap][8]
    float* rec_target;        // [cap]
    unsigned long long* rec_key;   // [cap]: traj << 28 | step << 14 | candidate
    uint32_t* rec_group;      // [cap]: index within the step's pairs << 16 | their count
    unsigned long long* rec_count;  // [2]: slots claimed, end of the filled prefix
    unsigned long long rec_cap;
};

// bytes of a trajectory state kept in a global slot (uint32 active lists)
inline size_t global_state_bytes(int n, int real_bytes, bool lists)
{
    const TreeGeom G = tree_geom(n);
    size_t b = align_up((size_t)((2 * n + 7) & ~7) * 2, 16) + align_up((size_t)G.total * 4, 16);
    b += 2 * align_up((size_t)n * real_bytes, 16);
    if (lists) b += 2 * align_up((size_t)n * 4, 16);
    return b;
}

// shared-memory sizes used by the plan
inline int group_state_bytes(int n, int64_t m, int real_bytes, bool rc_smem, bool lists, bool learned,
                             bool dm_smem)
{
    const TreeGeom G = tree_geom(n);
    size_t b = align_up((size_t)((2 * n + 7) & ~7) * 2, 16) + align_up((size_t)G.total * 4, 16);
    if (rc_smem) b += 2 * align_up((size_t)n * real_bytes, 16);
    if (lists) b += 2 * align_up((size_t)n * 2, 16);
    if (dm_smem) b += align_up((size_t)dm_ws_ints(n) * 4, 16) + align_up((size_t)m, 16);
    if (learned) b += 32 * 24 * 2;  // feature tile [32][24] bf16
    b += kGroupMiscInts * 4;
    return (int)b;
}

inline int staged_matrix_bytes(int n, int64_t m, bool with_ce)
{
    size_t b = 2 * align_up((size_t)(n + 1) * 4, 16) + 2 * align_up((size_t)m * 2, 16);
    if (with_ce) b += align_up((size_t)m * 4, 16);
    return (int)b;
}

struct StatsPartial {
    double c;          // max log x of the chunk (-inf if none alive)
    double s1, s2, m2; // sum y, sum y^2, sum (y - mean)^2 with y = exp(lx - c)
    unsigned long long cnt, alive;
};

struct StatsOut {
    double log_estimate, ess, p_match, rel_spread, rse, log_sum_x, log_sum_x2;
    unsigned long long n, alive;
};

// ---- launchers (pm_kernels.cu) ----
cudaError_t launch_prepare(DevMatrix* d_mats, const DevInput* d_in, int count, Sched s, int64_t m_max,
                           int n_max, uint32_t* status, cudaStream_t st);
cudaError_t launch_trajectories(const TrajParams& p, int grid, int smem_bytes, bool trace, cudaStream_t st);
cudaError_t launch_stats(const double* log_x, const uint64_t* h_prefix, const uint64_t* d_prefix,
                         int count, StatsPartial* partials, int chunks_per_matrix, StatsOut* out,
                         cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t count, uint32_t* out,
                          cudaStream_t st);
int traj_max_smem_bytes();
// PM_DEBUG build: out-of-range accesses the trajectory kernels' checked
// matrix views counted since the last call (the count is cleared); 0 in
// release builds
unsigned int traj_bounds_hits();
// on-chip bandwidth probes (pm_probe.cu)
cudaError_t launch_l2_probe(const void* buf, size_t bytes, int iters, int grid, unsigned long long* sink,
                            cudaStream_t st);
cudaError_t launch_smem_probe(int smem_bytes, int iters, int grid, unsigned long long* sink, cudaStream_t st);
// the kernel launch_trajectories would launch for these parameters (to find
// its node in a captured graph)
const void* traj_kernel_entry(const TrajParams& p, bool trace);
// learned proposal (pm_learn.cu)
int model_image_bytes();
int model_infer_bytes();
int model_param_count();
cudaError_t launch_model_image(const float* master, void* img, cudaStream_t st);
// group == nullptr: mean squared error; else the per-step centred loss (resid:
// device scratch of B floats for the batch's residuals)
// work: device scratch of mlp_grad_workspace_bytes(sm_count): its first int
// is the device error flag (the caller zeroes it once and reads it after the
// last launch; nonzero: a tensor-core completion wait ran out), then per-CTA
// partial sums, reduced in a fixed order so the gradient is reproducible
size_t mlp_grad_workspace_bytes(int sm_count);
cudaError_t launch_mlp_grad(const void* img, const float* feat, const float* target, const int* perm, int64_t row0,
                            int B, const uint32_t* group, float* resid, float* grad, double* loss, int sm_count,
                            void* work, cudaStream_t st);
cudaError_t launch_mlp_forward(const void* img, const float* feat, int B, float* out, int sm_count, cudaStream_t st);
cudaError_t launch_adam(float* master, float* m1, float* m2, const float* grad, float lr, float b1, float b2, float eps,
                        int step, void* img, cudaStream_t st);

}  // namespace pm
