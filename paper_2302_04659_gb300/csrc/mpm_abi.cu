// mpm_abi.cu -- the C-ABI of include/mpm.h: argument checks, workspace layout, the environment table,
// the per-substep launch sequence (optionally replayed from a CUDA graph) and the readbacks. All device
// memory comes from the caller's workspace; the library owns only the host handle and a small pinned
// staging buffer for collider uploads.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mpm.h"
#include "mpm_internal.h"
#include "mpm_net.h"

using namespace mpm;

namespace {
thread_local char g_last_error[256] = "";
}  // namespace

mpm_status mpm::record_cuda_error(cudaError_t e, const char* what) {
    snprintf(g_last_error, sizeof g_last_error, "%s: %s", what, cudaGetErrorString(e));
    return MPM_ERR_CUDA;
}

namespace mpm {

mpm_status check_material(const mpm_material* m) {
    if (!m) return MPM_ERR_INVALID_ARG;
    if (m->kind != MPM_PLASTICINE && m->kind != MPM_FLUID) return MPM_ERR_INVALID_ARG;
    if (!(m->rho > 0.0f) || !(m->p_vol > 0.0f)) return MPM_ERR_INVALID_ARG;
    if (m->kind == MPM_PLASTICINE) {
        if (!(m->E > 0.0f) || !(m->nu >= 0.0f && m->nu < 0.5f) || !(m->yield_stress >= 0.0f))
            return MPM_ERR_INVALID_ARG;
    } else {
        if (!(m->bulk_modulus >= 0.0f)) return MPM_ERR_INVALID_ARG;
    }
    return MPM_OK;
}

}  // namespace mpm

namespace {

mpm_status cuda_fail(cudaError_t e, const char* what) { return record_cuda_error(e, what); }

#define MPM_CUDA(call, what)                               \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

#define MPM_TRY(call)                \
    do {                             \
        mpm_status r_ = (call);      \
        if (r_ != MPM_OK) return r_; \
    } while (0)

constexpr size_t kAlign = 256;
constexpr int kMaxGraphs = 8;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Totals {
    size_t particles = 0, nodes = 0, bins = 0, colliders = 0;
};

Totals totals_of(int nenv, const mpm_env* envs) {
    Totals t;
    for (int e = 0; e < nenv; ++e) {
        const size_t nb = (size_t)envs[e].n / 4;
        t.particles += (size_t)envs[e].max_particles;
        t.bins += nb * nb * nb;
        t.nodes += nb * nb * nb * kBlkNodes;
        t.colliders += (size_t)envs[e].max_colliders;
    }
    return t;
}

struct Layout {
    size_t state[2], key, perm, grid[2], flags[2], hist, list[2], list_meta, cursor, chunks, tile_sums, envs,
        bin_env, colliders, poses, wrench, counters, sur, sur_reduce, total;
};

// Chunk list capacity: chunks of at least 32 particles, plus one partial chunk per bin.
size_t chunk_entries(const Totals& T) { return std::max<size_t>(T.particles, 1) / 32 + T.bins + 1; }

Layout make_layout(const Totals& T, int nenv) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align_up(bytes);
        return o;
    };
    const size_t cap = std::max<size_t>(T.particles, 1), kcap = std::max<size_t>(T.colliders, 1);
    for (int i = 0; i < 2; ++i) L.state[i] = take(cap * 25 * 4);
    L.key = take(cap * 8);  // (bin, rank within bin) per particle
    L.perm = take(cap * 4);
    for (int i = 0; i < 2; ++i) L.grid[i] = take(T.nodes * sizeof(float4));
    for (int i = 0; i < 2; ++i) L.flags[i] = take(T.bins * 4);
    L.hist = take(T.bins * 4 + 16);
    for (int i = 0; i < 2; ++i) L.list[i] = take(T.bins * 4);
    L.list_meta = take(4 * sizeof(uint32_t));  // list counts [2], grid-update CTAs done, spare
    // everything from grid[0] up to here restarts from zero on mpm_set_particles
    L.cursor = take(T.bins * 4 + 16);
    L.chunks = take(chunk_entries(T) * sizeof(int4));
    L.tile_sums = take(((T.bins + kScanTile - 1) / kScanTile + 1) * sizeof(uint2));
    L.envs = take((size_t)nenv * sizeof(EnvDesc));
    L.bin_env = take(T.bins * 4 + 16);  // padded to a multiple of 4 bins, like the counts
    L.colliders = take(kcap * sizeof(ColliderSet));  // written in stream order by each upload
    L.poses = take((kcap > (size_t)kSharedPoses ? (size_t)kPoseSteps * kcap : 1) * sizeof(ColliderNow));
    L.wrench = take(kcap * 6 * sizeof(double));
    L.counters = take(8 * sizeof(uint32_t));  // status, substep counter, num_chunks, fused-pass CTAs done,
                                              // fused-pass chunk counter, sort-assign CTAs done, spare
    // surrogate window: sums, box, gate word, stats, the wrench before the window
    L.sur = take(16 * sizeof(double) + 8 * sizeof(int) + 8 * sizeof(double) + kcap * 6 * sizeof(double));
    L.sur_reduce = take((size_t)kReduceBlocks * 4 * sizeof(Pair) + 16);  // per-block totals, ticket
    L.total = off;
    return L;
}


mpm_status check_batch(const mpm_config* c, int nenv, const mpm_env* envs) {
    if (!c || !envs || nenv < 1 || nenv > MPM_MAX_ENVS) return MPM_ERR_INVALID_ARG;
    if (!(c->dt > 0.0f) || !std::isfinite(c->dt)) return MPM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(c->gravity[a])) return MPM_ERR_INVALID_ARG;
    if (c->bound < 0) return MPM_ERR_INVALID_ARG;
    size_t particles = 0;
    for (int e = 0; e < nenv; ++e) {
        const mpm_env& v = envs[e];
        if (v.n < 8 || v.n > 256 || (v.n % 4) != 0) return MPM_ERR_INVALID_ARG;
        if (2 * c->bound > v.n) return MPM_ERR_INVALID_ARG;
        if (v.max_particles < 1 || v.max_colliders < 0 || v.max_colliders > MPM_MAX_COLLIDERS) return MPM_ERR_INVALID_ARG;
        MPM_TRY(check_material(&v.material));
        particles += (size_t)v.max_particles;
    }
    if (particles > (size_t)(1 << 30)) return MPM_ERR_INVALID_ARG;
    return MPM_OK;
}

mpm_env env_from_single(const mpm_config* cfg, const mpm_material* mat) {
    mpm_env e{};
    e.n = cfg->n;
    e.max_particles = cfg->max_particles;
    e.max_colliders = cfg->max_colliders;
    e.material = *mat;
    return e;
}

// Host-side pipeline state that the enqueued work depends on (and that a cached graph assumes).
struct PipeState {
    int cur = 0;               // state buffer holding the current particles
    int g = 0;                 // grid holding the particle-to-grid transfer of the current state
    bool scanned = false;      // bin offsets and chunk list match the current keys
    bool order_valid = false;  // perm (sorted slot -> particle) matches them too
    bool grid_valid = false;   // grid g holds the transfer of the current state
    bool rechunk = false;      // the chunk size changed since the scan: recut the chunk list
    bool counts_pending = false;  // the bin counts of the current keys are in hist, not yet scanned
    bool operator==(const PipeState& o) const {
        return cur == o.cur && g == o.g && scanned == o.scanned && order_valid == o.order_valid &&
               grid_valid == o.grid_valid && rechunk == o.rechunk && counts_pending == o.counts_pending;
    }
};

struct TimedNode {  // an event-record node of a cached graph bracketing one launch
    cudaGraphNode_t start, stop;
    int kind;
};

struct GraphEntry {
    int n_substeps, N, ncol;
    unsigned timing_mask;
    PipeState before, after;
    long long launches;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    std::vector<TimedNode> timed;
    unsigned long long last_use;
};

}  // namespace

struct mpm_sim {
    mpm_config cfg;
    int nenv = 0;
    int kind_all = 0;  // the material of every env, -1 if they differ
    std::vector<mpm_env> env_cfg;
    std::vector<EnvDesc> envs;  // host copy of the device table
    Totals T;
    Layout L;
    char* ws = nullptr;
    int N = 0;  // particles of all envs
    PipeState ps;
    std::vector<mpm_shape> shapes;
    std::vector<int> shape_counts;  // shapes per env
    int ncol = 0;  // colliders uploaded by the last mpm_set_colliders
    int contact = MPM_CONTACT_GRID;  // mpm_set_contact
    float stiffness = 0.0f, damping = 0.0f;
    bool sur_pending = false;  // a surrogate window was started and not yet ended
    // attached surrogate network (mpm_surrogate_attach)
    bool net_attached = false;
    long long sur_steps_redone = 0, sur_windows_redone = 0;
    // the box of the next surrogate step, computed with the previous step's readback
    bool box_cached = false;
    mpm_box box_cache{};
    PipeState box_cache_ps;
    long long box_cache_version = 0;
    int box_cache_n = 0;
    long long particles_version = 0;  // bumped by every particle upload
    // a gated surrogate step awaiting its verdict (resolved by the next call that depends on the state)
    bool verify_pending = false;
    cudaEvent_t verify_event = nullptr;
    uint32_t* verify_host = nullptr;   // pinned: the gate's word, then the next box (6 ints)
    int verify_substeps = 0;
    cudaStream_t verify_stream = nullptr;
    PipeState verify_ps;               // the state the step ended in (for the next box)
    long long upload_seq = 0, verify_upload_seq = 0;
    ColliderUpload last_upload{};      // the latest collider upload (at most kSharedPoses bodies)
    mpm_surrogate_net net{};
    char* net_ws = nullptr;
    int net_max_voxels = 0;
    std::vector<GraphEntry> sur_graphs;
    std::vector<std::array<int, 8>> sur_keys;  // box (6), substeps, gate of each cached graph
    ColliderSet* stage = nullptr;  // pinned staging for collider uploads
    cudaEvent_t stage_done = nullptr;
    int sms = 0;
    int chunk = kChunk, fused_cps = 1, grid_cps = 2, p2g_cps = 1, max_fused_cps = 1;
    long long launches = 0;
    unsigned timing_mask = 0;
    struct Ev {
        cudaEvent_t a, b;
        int kind;
    };
    std::vector<Ev> pending;
    std::vector<cudaEvent_t> pool;
    double ms[MPM_K_COUNT] = {};
    long long counts[MPM_K_COUNT] = {};
    // graph capture and replay of mpm_substep
    bool use_graphs = true;
    bool capturing = false;
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphEntry> graphs;
    std::vector<std::pair<cudaEvent_t, int>> cap_events;  // (event, kind), start/stop alternating
    unsigned long long use_clock = 0;

    template <class T>
    T* at(size_t off) {
        return reinterpret_cast<T*>(ws + off);
    }
    uint32_t* status() { return at<uint32_t>(L.counters); }
    uint32_t* substep_counter() { return at<uint32_t>(L.counters) + 1; }
    uint32_t* num_chunks() { return at<uint32_t>(L.counters) + 2; }
    uint32_t* done() { return at<uint32_t>(L.counters) + 3; }
    uint32_t* work() { return at<uint32_t>(L.counters) + 4; }
    uint32_t* scan_done() { return at<uint32_t>(L.counters) + 5; }
    uint32_t* list(int which) { return at<uint32_t>(L.list[which]); }
    uint32_t* list_count(int which) { return at<uint32_t>(L.list_meta) + which; }
    uint32_t* grid_done() { return at<uint32_t>(L.list_meta) + 2; }
    double* sur_sums() { return at<double>(L.sur); }  // a window's kSumWindow sums, then 3 spare at [12..15)
    int* sur_box() { return reinterpret_cast<int*>(at<char>(L.sur) + 16 * sizeof(double)); }
    uint32_t* sur_gate() { return at<uint32_t>(L.sur + 16 * sizeof(double) + 6 * sizeof(int)); }
    unsigned long long* sur_stats() { return at<unsigned long long>(L.sur + 16 * sizeof(double) + 8 * sizeof(int)); }
    double* sur_wrench() { return at<double>(L.sur + 16 * sizeof(double) + 8 * sizeof(int) + 8 * sizeof(double)); }
    ReduceScratch sur_reduce() {
        return ReduceScratch{at<Pair>(L.sur_reduce),
                             reinterpret_cast<uint32_t*>(at<char>(L.sur_reduce) + (size_t)kReduceBlocks * 4 * sizeof(Pair))};
    }
    const EnvDesc* envs_dev() { return at<EnvDesc>(L.envs); }
    bool tail_scan() const { return T.bins <= (size_t)kTailScanMaxBins; }
    StateView view(int which) {
        float* b = at<float>(L.state[which]);
        const size_t n = (size_t)N;
        StateView s;
        s.x = b;
        s.v = b + 3 * n;
        s.C = b + 6 * n;
        s.F = b + 15 * n;
        s.pid = reinterpret_cast<uint32_t*>(b + 24 * std::max<size_t>(T.particles, 1));
        return s;
    }
    cudaEvent_t get_event() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    void drop_graphs() {
        for (auto* list : {&graphs, &sur_graphs})
            for (auto& ge : *list) {
                cudaGraphExecDestroy(ge.exec);
                cudaGraphDestroy(ge.graph);
            }
        graphs.clear();
        sur_graphs.clear();
        sur_keys.clear();
    }
};

namespace {

// Enqueue one launch; bracket it with timing events when its kind is selected. While capturing a graph
// the events become event-record nodes whose events are swapped on every replay.
template <class F>
mpm_status launch(mpm_sim* s, int kind, cudaStream_t st, F&& fn, const char* what) {
    const bool timed = (s->timing_mask >> kind) & 1u;
    cudaEvent_t a = nullptr, b = nullptr;
    if (timed) {
        a = s->get_event();
        b = s->get_event();
        if (s->capturing)
            MPM_CUDA(cudaEventRecordWithFlags(a, st, cudaEventRecordExternal), "cudaEventRecordWithFlags");
        else
            MPM_CUDA(cudaEventRecord(a, st), "cudaEventRecord");
    }
    MPM_CUDA(fn(), what);
    ++s->launches;
    if (timed) {
        if (s->capturing) {
            MPM_CUDA(cudaEventRecordWithFlags(b, st, cudaEventRecordExternal), "cudaEventRecordWithFlags");
            s->cap_events.push_back({a, kind});
            s->cap_events.push_back({b, kind});
        } else {
            MPM_CUDA(cudaEventRecord(b, st), "cudaEventRecord");
            s->pending.push_back({a, b, kind});
        }
    }
    return MPM_OK;
}

mpm_status upload_envs(mpm_sim* s, cudaStream_t st) {
    MPM_CUDA(cudaMemcpyAsync(s->at<EnvDesc>(s->L.envs), s->envs.data(), sizeof(EnvDesc) * s->nenv,
                             cudaMemcpyHostToDevice, st),
             "copy env table");
    return MPM_OK;
}

TransferParams transfer_params(mpm_sim* s) {
    TransferParams p{};
    p.envs = s->envs_dev();
    p.env0 = s->envs[0];
    p.one_env = s->nenv == 1 ? 1 : 0;
    p.kind_all = s->kind_all;
    p.N = s->N;
    p.in = s->view(s->ps.cur);
    p.out = s->view(1 - s->ps.cur);
    p.perm = s->at<uint32_t>(s->L.perm);
    p.keyrank_out = s->at<uint2>(s->L.key);
    p.hist = s->at<uint32_t>(s->L.hist);
    p.chunks = s->at<int4>(s->L.chunks);
    p.num_chunks = s->num_chunks();
    p.chunk_cap = (int)chunk_entries(s->T);
    p.status = s->status();
    p.substep_counter = s->substep_counter();
    p.tail_scan = s->tail_scan() ? 1 : 0;
    p.total_bins = (int)s->T.bins;
    p.chunk = s->chunk;
    p.bin_env = s->nenv > 1 ? s->at<uint32_t>(s->L.bin_env) : nullptr;  // null: all bins are env 0's
    p.cursor = s->at<uint32_t>(s->L.cursor);
    p.chunks_next = s->at<int4>(s->L.chunks);
    p.num_chunks_next = s->num_chunks();
    p.done = s->done();
    p.work = s->work();
    p.contact = s->contact == MPM_CONTACT_PARTICLE ? 1 : 0;
    p.stiffness = s->stiffness;
    p.damping = s->damping;
    p.cols = s->at<ColliderSet>(s->L.colliders);
    p.poses = s->at<ColliderNow>(s->L.poses);
    p.k_total = s->ncol;
    p.wrench = s->at<double>(s->L.wrench);
    p.scatter = 1;
    return p;
}

GridParams grid_params(mpm_sim* s) {
    GridParams gp{};
    gp.envs = s->envs_dev();
    gp.env0 = s->envs[0];
    gp.one_env = s->nenv == 1 ? 1 : 0;
    gp.dt = s->cfg.dt;
    for (int a = 0; a < 3; ++a) gp.gravity[a] = s->cfg.gravity[a];
    gp.bound = s->cfg.bound;
    gp.grid = s->at<float4>(s->L.grid[s->ps.g]);
    gp.list = s->list(s->ps.g);
    gp.list_count = s->list_count(s->ps.g);
    gp.list_cap = (int)s->T.bins;
    gp.grid_old = s->at<float4>(s->L.grid[1 - s->ps.g]);
    gp.flags_old = s->at<uint32_t>(s->L.flags[1 - s->ps.g]);
    gp.list_old = s->list(1 - s->ps.g);
    gp.list_count_old = s->list_count(1 - s->ps.g);
    gp.done = s->grid_done();
    gp.cols = s->at<ColliderSet>(s->L.colliders);
    gp.poses = s->at<ColliderNow>(s->L.poses);
    gp.k_total = s->ncol;  // also the row stride of the pose table mpm_set_colliders fills
    gp.substep_counter = s->substep_counter();
    gp.wrench = s->at<double>(s->L.wrench);
    gp.ctas = (int)std::max<size_t>(1, std::min<size_t>((size_t)s->sms * s->grid_cps, (s->T.bins + 3) / 4));
    gp.grid_colliders = s->contact == MPM_CONTACT_GRID ? 1 : 0;
    return gp;
}

ScanParams scan_params(mpm_sim* s) {
    ScanParams sp{};
    sp.hist = s->at<uint32_t>(s->L.hist);
    sp.cursor = s->at<uint32_t>(s->L.cursor);
    sp.chunks = s->at<int4>(s->L.chunks);
    sp.num_chunks = s->num_chunks();
    sp.tile_sums = s->at<uint2>(s->L.tile_sums);
    sp.bin_env = s->at<uint32_t>(s->L.bin_env);
    sp.total_bins = (int)s->T.bins;
    sp.chunk = s->chunk;
    return sp;
}

mpm_status enqueue_scan(mpm_sim* s, cudaStream_t st) {
    if (s->tail_scan()) {
        return launch(s, MPM_K_SCAN, st, [&] {
            return launch_scan_binned(s->at<uint32_t>(s->L.hist), s->at<uint32_t>(s->L.cursor),
                                      s->at<int4>(s->L.chunks), s->num_chunks(),
                                      s->nenv > 1 ? s->at<uint32_t>(s->L.bin_env) : nullptr, (int)s->T.bins,
                                      s->chunk, st);
        }, "scan");
    }
    ScanParams sp = scan_params(s);
    return launch(s, MPM_K_SCAN, st, [&] { return launch_scan_grid(sp, st); }, "scan_grid");
}

mpm_status ensure_scanned(mpm_sim* s, cudaStream_t st) {
    if (s->ps.scanned && !s->ps.rechunk) return MPM_OK;
    if (s->ps.rechunk) {  // the bins' counts again, from their offsets, for a scan with the new chunk size
        MPM_TRY(launch(s, MPM_K_SCAN, st, [&] {
            return launch_hist_from_cursor(s->at<uint32_t>(s->L.cursor), s->at<uint32_t>(s->L.hist), (int)s->T.bins,
                                           (uint32_t)s->N, st);
        }, "hist_from_cursor"));
        s->ps.rechunk = false;
    }
    MPM_TRY(enqueue_scan(s, st));
    s->ps.scanned = true;
    s->ps.counts_pending = false;
    return MPM_OK;
}

mpm_status ensure_order(mpm_sim* s, cudaStream_t st) {
    MPM_TRY(ensure_scanned(s, st));
    if (s->ps.order_valid) return MPM_OK;
    MPM_TRY(launch(s, MPM_K_ASSIGN, st, [&] {
        return launch_assign(s->N, s->at<uint2>(s->L.key), s->at<uint32_t>(s->L.cursor), s->at<uint32_t>(s->L.perm),
                             st);
    }, "assign"));
    s->ps.order_valid = true;
    return MPM_OK;
}

// Particle-to-grid transfer of the current state into grid g (only after the state was replaced).
mpm_status ensure_grid(mpm_sim* s, cudaStream_t st) {
    if (s->ps.grid_valid) return MPM_OK;
    MPM_TRY(ensure_order(s, st));
    TransferParams p = transfer_params(s);
    p.grid_out = s->at<float4>(s->L.grid[s->ps.g]);
    p.flags_out = s->at<uint32_t>(s->L.flags[s->ps.g]);
    p.list_out = s->list(s->ps.g);
    p.list_count_out = s->list_count(s->ps.g);
    MPM_TRY(launch(s, MPM_K_P2G, st, [&] { return launch_p2g(p, s->sms * s->p2g_cps, st); }, "p2g"));
    s->ps.grid_valid = true;
    return MPM_OK;
}

// First half of a substep: the sort-assign of the current state and the grid update of its transfer.
mpm_status enqueue_grid_half(mpm_sim* s, cudaStream_t st, const uint32_t* gate = nullptr, uint32_t gate_run = 1,
                             double* p0_sums = nullptr) {
    // the fused pass left its bin counts unscanned: the sort-assign CTAs of this launch scan them
    const bool scan_here = s->ps.counts_pending && !s->ps.rechunk && !gate && s->ps.grid_valid && s->tail_scan();
    if (!scan_here) MPM_TRY(ensure_scanned(s, st));
    MPM_TRY(ensure_grid(s, st));
    AssignGridParams ap{};
    if (scan_here) {
        ap.scan = 1;
        ap.hist = s->at<uint32_t>(s->L.hist);
        ap.cursor_out = s->at<uint32_t>(s->L.cursor);
        ap.chunks = s->at<int4>(s->L.chunks);
        ap.num_chunks = s->num_chunks();
        ap.bin_env = s->nenv > 1 ? s->at<uint32_t>(s->L.bin_env) : nullptr;
        ap.total_bins = (int)s->T.bins;
        ap.chunk = s->chunk;
        ap.scan_done = s->scan_done();
        ap.status = s->status();
        s->ps.scanned = true;
        s->ps.counts_pending = false;
    }
    ap.gate = gate;
    ap.gate_run = gate_run;
    ap.grid = grid_params(s);
    ap.grid.p0_sums = p0_sums;
    ap.N = s->N;
    ap.keyrank = s->at<uint2>(s->L.key);
    ap.cursor = s->at<uint32_t>(s->L.cursor);
    ap.perm = s->at<uint32_t>(s->L.perm);
    ap.assign_ctas = s->ps.order_valid ? 0 : (s->N + 1023) / 1024;  // 4 particles per thread
    if (scan_here) {  // fewer, longer sort-assign CTAs (each scans the counts once); at least one, to clear them
        ap.assign_ctas = std::max(1, (s->N + 1024 * kScanAssignRounds - 1) / (1024 * kScanAssignRounds));
    }
    MPM_TRY(launch(s, MPM_K_GRID, st, [&] { return launch_assign_grid(ap, st); }, "assign_grid"));
    s->ps.order_valid = true;
    return MPM_OK;
}

// Second half: the fused G2P -> P2G pass from the updated grid (advecting by advect_dt, the substep's dt
// unless a surrogate window overrides it for a one-env handle), then the bin scan if it is separate.
mpm_status enqueue_particle_half(mpm_sim* s, cudaStream_t st, float advect_dt = 0.0f, const uint32_t* gate = nullptr,
                                 uint32_t gate_run = 1, bool scatter = true) {
    TransferParams p = transfer_params(s);
    p.scatter = scatter ? 1 : 0;
    p.gate = gate;
    p.gate_run = gate_run;
    p.grid_in = s->at<float4>(s->L.grid[s->ps.g]);
    p.grid_out = s->at<float4>(s->L.grid[1 - s->ps.g]);
    p.flags_out = s->at<uint32_t>(s->L.flags[1 - s->ps.g]);
    p.list_out = s->list(1 - s->ps.g);
    p.list_count_out = s->list_count(1 - s->ps.g);
    if (advect_dt > 0.0f) p.env0.geo.dt = advect_dt;
    // Plain substeps with few bins leave the new counts for the next grid-half launch to scan; a gated
    // window's launch (both branches enqueued, one runs) scans at the end of the fused pass as before.
    const bool defer = s->tail_scan() && !gate && scatter;
    if (defer) p.tail_scan = 0;
    MPM_TRY(launch(s, MPM_K_G2P2G, st, [&] { return launch_g2p2g(p, s->sms * s->fused_cps, st); }, "g2p2g"));
    s->ps.cur = 1 - s->ps.cur;
    s->ps.g = 1 - s->ps.g;
    s->ps.order_valid = false;  // assigned by the next launch
    s->ps.grid_valid = scatter;
    s->ps.counts_pending = defer;
    if (defer) s->ps.rechunk = false;  // the pending counts are cut with the current chunk size
    s->ps.scanned = s->tail_scan() && !defer;  // the fused pass's last CTA wrote the new bins
    if (!s->ps.scanned && !defer) MPM_TRY(ensure_scanned(s, st));
    return MPM_OK;
}

// The launches of n substeps: per substep one sort-assign + grid-update launch and one fused
// G2P->P2G launch (whose last CTA sorts the new positions into bins; with many bins two scan launches
// follow instead). With the particle form of the contact the last fused launch stops after G2P: the
// next call's first transfer then takes its penalties at the poses set in between.
mpm_status enqueue_substeps(mpm_sim* s, int n, cudaStream_t st) {
    const bool particle_contact = s->contact == MPM_CONTACT_PARTICLE;
    for (int it = 0; it < n; ++it) {
        MPM_TRY(enqueue_grid_half(s, st));
        MPM_TRY(enqueue_particle_half(s, st, 0.0f, nullptr, 1, !(particle_contact && it == n - 1)));
    }
    return MPM_OK;
}

// Capture the launches of n substeps from the current pipeline state into a graph.
mpm_status capture_graph(mpm_sim* s, int n, GraphEntry& ge) {
    if (!s->cap_stream) MPM_CUDA(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate");
    ge.n_substeps = n;
    ge.N = s->N;
    ge.ncol = s->ncol;
    ge.timing_mask = s->timing_mask;
    ge.before = s->ps;
    const long long l0 = s->launches;
    s->cap_events.clear();
    MPM_CUDA(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    s->capturing = true;
    mpm_status r = enqueue_substeps(s, n, s->cap_stream);
    s->capturing = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s->cap_stream, &graph);
    // the host-side state after the captured sequence is the state after every replay of it
    ge.after = s->ps;
    ge.launches = s->launches - l0;
    s->ps = ge.before;
    s->launches = l0;
    if (r != MPM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return r;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    ge.graph = graph;
    ge.exec = exec;
    // event-record nodes, matched to the capture order
    size_t count = 0;
    MPM_CUDA(cudaGraphGetNodes(graph, nullptr, &count), "cudaGraphGetNodes");
    std::vector<cudaGraphNode_t> nodes(count);
    if (count) MPM_CUDA(cudaGraphGetNodes(graph, nodes.data(), &count), "cudaGraphGetNodes");
    std::vector<cudaGraphNode_t> by_event(s->cap_events.size(), nullptr);
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        MPM_CUDA(cudaGraphNodeGetType(nd, &t), "cudaGraphNodeGetType");
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        MPM_CUDA(cudaGraphEventRecordNodeGetEvent(nd, &ev), "cudaGraphEventRecordNodeGetEvent");
        for (size_t i = 0; i < s->cap_events.size(); ++i)
            if (s->cap_events[i].first == ev) by_event[i] = nd;
    }
    for (size_t i = 0; i + 1 < s->cap_events.size(); i += 2) {
        if (!by_event[i] || !by_event[i + 1]) continue;
        ge.timed.push_back({by_event[i], by_event[i + 1], s->cap_events[i].second});
    }
    for (auto& pe : s->cap_events) s->pool.push_back(pe.first);
    s->cap_events.clear();
    return MPM_OK;
}

GraphEntry* find_graph(mpm_sim* s, int n) {
    for (auto& ge : s->graphs)
        if (ge.n_substeps == n && ge.N == s->N && ge.ncol == s->ncol && ge.timing_mask == s->timing_mask &&
            ge.before == s->ps)
            return &ge;
    return nullptr;
}

mpm_status create_impl(const mpm_config* cfg, int nenv, const mpm_env* envs, void* d_workspace, size_t bytes,
                       void* stream, mpm_sim** out) {
    if (!out) return MPM_ERR_INVALID_ARG;
    *out = nullptr;
    MPM_TRY(check_batch(cfg, nenv, envs));
    const Totals T = totals_of(nenv, envs);
    const Layout L = make_layout(T, nenv);
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) % kAlign) != 0 || bytes < L.total)
        return MPM_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mpm_sim* s = new (std::nothrow) mpm_sim();
    if (!s) return MPM_ERR_INVALID_ARG;
    s->cfg = *cfg;
    s->nenv = nenv;
    s->env_cfg.assign(envs, envs + nenv);
    s->T = T;
    s->L = L;
    s->ws = static_cast<char*>(d_workspace);
    s->envs.resize(nenv);
    std::vector<uint32_t> bin_env(T.bins);
    uint32_t bin_base = 0, node_base = 0;
    for (int e = 0; e < nenv; ++e) {
        const mpm_env& v = envs[e];
        EnvDesc& d = s->envs[e];
        d = EnvDesc{};
        Geometry& g = d.geo;
        g.n = v.n;
        g.nb = v.n / 4;
        g.nblocks = g.nb * g.nb * g.nb;
        g.nb_recip = 0xFFFFFFFFu / (uint32_t)g.nb + 1u;
        g.dx = (float)(1.0 / v.n);
        g.inv_dx = (float)v.n;
        g.dt = cfg->dt;
        g.lo = (float)(2.0 / v.n);
        g.hi = (float)(1.0 - 2.0 / v.n);
        const mpm_material& m = v.material;
        double mu = 0.0, lambda = m.bulk_modulus;
        if (m.kind == MPM_PLASTICINE) {
            mu = (double)m.E / (2.0 * (1.0 + m.nu));
            lambda = (double)m.E * m.nu / ((1.0 + m.nu) * (1.0 - 2.0 * m.nu));
        }
        d.mat.mu = (float)mu;
        d.mat.lambda = (float)lambda;
        d.mat.yield_radius = mu > 0.0 ? (float)(m.yield_stress / (2.0 * mu)) : 0.0f;
        d.mat.p_mass = (float)((double)m.rho * m.p_vol);
        d.mat.stress_scale = (float)(-(double)cfg->dt * m.p_vol * 4.0 * v.n * v.n);
        d.kind = m.kind;
        d.bin_base = bin_base;
        d.node_base = node_base;
        for (int b = 0; b < g.nblocks; ++b) bin_env[bin_base + b] = (uint32_t)e;
        bin_base += (uint32_t)g.nblocks;
        node_base += (uint32_t)g.nblocks * kBlkNodes;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&s->stage),
                                            std::max<size_t>(T.colliders, 1) * sizeof(ColliderSet), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->stage_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->ws + L.grid[0], 0, L.total - L.grid[0], st);
    if (e == cudaSuccess && T.bins)
        e = cudaMemcpyAsync(s->at<uint32_t>(L.bin_env), bin_env.data(), T.bins * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->at<EnvDesc>(L.envs), s->envs.data(), sizeof(EnvDesc) * nenv, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host tables above are temporaries
    if (e != cudaSuccess) {
        mpm_status r = cuda_fail(e, "create");
        mpm_destroy(s);
        return r;
    }
    s->kind_all = envs[0].material.kind;
    for (int e = 1; e < nenv; ++e)
        if (envs[e].material.kind != s->kind_all) s->kind_all = -1;
    s->chunk = nenv == 1 ? kChunk : 128;  // dense single scenes: 256-particle chunks; batches: 128
    s->max_fused_cps = transfer_ctas_per_sm(true, s->kind_all, nenv == 1, false, s->chunk);
    s->fused_cps = s->max_fused_cps;
    s->p2g_cps = transfer_ctas_per_sm(false, s->kind_all, nenv == 1);
    s->ps.scanned = s->ps.order_valid = s->ps.grid_valid = true;  // no particles yet
    *out = s;
    return MPM_OK;
}

}  // namespace

extern "C" {

static mpm_status resolve_pending(mpm_sim* s);

const char* mpm_status_string(mpm_status s) {
    switch (s) {
        case MPM_OK: return "ok";
        case MPM_ERR_INVALID_ARG: return "invalid argument";
        case MPM_ERR_CUDA: return "CUDA error";
        case MPM_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case MPM_ERR_CAPACITY: return "capacity exceeded";
    }
    return "unknown status";
}

const char* mpm_last_error(void) { return g_last_error; }

mpm_status mpm_workspace_size_batch(const mpm_config* cfg, int nenv, const mpm_env* envs, size_t* bytes) {
    if (!bytes) return MPM_ERR_INVALID_ARG;
    MPM_TRY(check_batch(cfg, nenv, envs));
    *bytes = make_layout(totals_of(nenv, envs), nenv).total;
    return MPM_OK;
}

mpm_status mpm_workspace_size(const mpm_config* cfg, const mpm_material* mat, size_t* bytes) {
    if (!cfg || !mat) return MPM_ERR_INVALID_ARG;
    const mpm_env e = env_from_single(cfg, mat);
    return mpm_workspace_size_batch(cfg, 1, &e, bytes);
}

mpm_status mpm_create_batch(const mpm_config* cfg, int nenv, const mpm_env* envs, void* d_workspace, size_t bytes,
                            void* stream, mpm_sim** out) {
    return create_impl(cfg, nenv, envs, d_workspace, bytes, stream, out);
}

mpm_status mpm_create(const mpm_config* cfg, const mpm_material* mat, void* d_workspace, size_t bytes, void* stream,
                      mpm_sim** out) {
    if (out) *out = nullptr;
    if (!cfg || !mat) return MPM_ERR_INVALID_ARG;
    const mpm_env e = env_from_single(cfg, mat);
    return create_impl(cfg, 1, &e, d_workspace, bytes, stream, out);
}

void mpm_destroy(mpm_sim* s) {
    if (!s) return;
    if (s->verify_event) {
        cudaEventSynchronize(s->verify_event);
        cudaEventDestroy(s->verify_event);
    }
    if (s->verify_host) cudaFreeHost(s->verify_host);
    s->drop_graphs();
    for (auto& ev : s->pending) {
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.b);
    }
    for (auto e : s->pool) cudaEventDestroy(e);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->stage_done) {
        cudaEventSynchronize(s->stage_done);
        cudaEventDestroy(s->stage_done);
    }
    if (s->stage) cudaFreeHost(s->stage);
    delete s;
}

int mpm_num_particles(const mpm_sim* s) { return s ? s->N : 0; }

int mpm_num_envs(const mpm_sim* s) { return s ? s->nenv : 0; }

long long mpm_launch_count(const mpm_sim* s) { return s ? s->launches : 0; }

mpm_status mpm_set_particles_batch(mpm_sim* s, const int* counts, const float* x, const float* v, const float* C,
                                   const float* F, int src_on_device, void* stream) {
    if (!s || !counts) return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    size_t total = 0;
    for (int e = 0; e < s->nenv; ++e) {
        if (counts[e] < 0) return MPM_ERR_INVALID_ARG;
        if (counts[e] > s->env_cfg[e].max_particles) return MPM_ERR_CAPACITY;
        total += (size_t)counts[e];
    }
    if (total > 0 && !x) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t first = 0;
    for (int e = 0; e < s->nenv; ++e) {
        s->envs[e].part_first = first;
        s->envs[e].part_count = (uint32_t)counts[e];
        first += (uint32_t)counts[e];
    }
    MPM_TRY(upload_envs(s, st));
    // grids, bin flags, lists and histogram restart from zero
    const size_t z0 = s->L.grid[0], z1 = s->L.cursor;
    MPM_CUDA(cudaMemsetAsync(s->ws + z0, 0, z1 - z0, st), "cudaMemsetAsync");
    s->N = (int)total;
    s->ps = PipeState{};
    s->sur_pending = false;
    s->particles_version += 1;
    if (total == 0) {
        s->ps.scanned = s->ps.order_valid = s->ps.grid_valid = true;
        return MPM_OK;
    }
    const size_t N = total;
    const float *sx = x, *sv = v, *sC = C, *sF = F;
    if (!src_on_device) {
        // stage host arrays in the spare state buffer, same SoA layout
        StateView stage = s->view(1);
        MPM_CUDA(cudaMemcpyAsync(stage.x, x, 3 * N * 4, cudaMemcpyHostToDevice, st), "copy x");
        sx = stage.x;
        if (v) {
            MPM_CUDA(cudaMemcpyAsync(stage.v, v, 3 * N * 4, cudaMemcpyHostToDevice, st), "copy v");
            sv = stage.v;
        }
        if (C) {
            MPM_CUDA(cudaMemcpyAsync(stage.C, C, 9 * N * 4, cudaMemcpyHostToDevice, st), "copy C");
            sC = stage.C;
        }
        if (F) {
            MPM_CUDA(cudaMemcpyAsync(stage.F, F, 9 * N * 4, cudaMemcpyHostToDevice, st), "copy F");
            sF = stage.F;
        }
    }
    LoadParams lp{};
    lp.envs = s->envs_dev();
    lp.nenv = s->nenv;
    lp.N = (int)N;
    lp.x = sx;
    lp.v = sv;
    lp.C = sC;
    lp.F = sF;
    lp.dst = s->view(0);
    lp.keyrank = s->at<uint2>(s->L.key);
    lp.hist = s->at<uint32_t>(s->L.hist);
    lp.status = s->status();
    MPM_TRY(launch(s, MPM_K_LOAD, st, [&] { return launch_load(lp, st); }, "load"));
    if (!src_on_device) MPM_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return MPM_OK;
}

mpm_status mpm_set_particles(mpm_sim* s, int n, const float* x, const float* v, const float* C, const float* F,
                             int src_on_device, void* stream) {
    if (!s || s->nenv != 1 || n < 0 || (n > 0 && !x)) return MPM_ERR_INVALID_ARG;
    return mpm_set_particles_batch(s, &n, x, v, C, F, src_on_device, stream);
}

mpm_status mpm_set_shapes_batch(mpm_sim* s, const int* counts, const mpm_shape* shapes) {
    if (!s || !counts) return MPM_ERR_INVALID_ARG;
    int total = 0;
    for (int e = 0; e < s->nenv; ++e) {
        if (counts[e] < 0) return MPM_ERR_INVALID_ARG;
        if (counts[e] > s->env_cfg[e].max_colliders) return MPM_ERR_CAPACITY;
        total += counts[e];
    }
    if (total > 0 && !shapes) return MPM_ERR_INVALID_ARG;
    for (int i = 0; i < total; ++i) {
        const mpm_shape& sh = shapes[i];
        if (sh.type != MPM_BOX && sh.type != MPM_CAPSULE && sh.type != MPM_SDF_VOLUME) return MPM_ERR_INVALID_ARG;
        if (!(sh.friction >= 0.0f) || !std::isfinite(sh.friction)) return MPM_ERR_INVALID_ARG;
        if (sh.type == MPM_SDF_VOLUME) {
            if (!sh.sdf || !(sh.sdf_h > 0.0f) || !std::isfinite(sh.sdf_h)) return MPM_ERR_INVALID_ARG;
            if (reinterpret_cast<uintptr_t>(sh.sdf) % alignof(float)) return MPM_ERR_INVALID_ARG;
            for (int a = 0; a < 3; ++a)
                if (sh.res[a] < 2 || sh.res[a] > 4096 || !std::isfinite(sh.sdf_origin[a])) return MPM_ERR_INVALID_ARG;
            continue;
        }
        const int dims = sh.type == MPM_BOX ? 3 : 2;
        for (int a = 0; a < dims; ++a)
            if (!(sh.half[a] >= 0.0f) || !std::isfinite(sh.half[a])) return MPM_ERR_INVALID_ARG;
    }
    s->shapes.assign(shapes, shapes + total);
    int first = 0;
    for (int e = 0; e < s->nenv; ++e) {
        s->envs[e].col_first = first;
        s->envs[e].col_count = 0;  // active after the next mpm_set_colliders
        first += counts[e];
    }
    s->shape_counts.assign(counts, counts + s->nenv);
    return MPM_OK;
}

mpm_status mpm_set_shapes(mpm_sim* s, int k, const mpm_shape* shapes) {
    if (!s || s->nenv != 1 || k < 0 || (k > 0 && !shapes)) return MPM_ERR_INVALID_ARG;
    if (k > s->env_cfg[0].max_colliders) return MPM_ERR_CAPACITY;
    return mpm_set_shapes_batch(s, &k, shapes);
}

mpm_status mpm_set_colliders(mpm_sim* s, int k, const float* pose, const float* lin_vel, const float* ang_vel,
                             const float* com, void* stream) {
    if (!s || k != (int)s->shapes.size() || (k > 0 && (!pose || !lin_vel))) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the previous upload must have left the staging buffer before it is refilled
    MPM_CUDA(cudaEventSynchronize(s->stage_done), "cudaEventSynchronize");
    for (int i = 0; i < k; ++i) {
        ColliderSet& c = s->stage[i];
        const mpm_shape& sh = s->shapes[i];
        c.type = sh.type;
        for (int a = 0; a < 3; ++a) c.half[a] = sh.half[a];
        c.friction = sh.friction;
        c.vol = SdfVolume{};
        double reach = 0.0;  // a ball about the frame origin holding the body: inside points lie in it
        if (sh.type == MPM_SDF_VOLUME) {
            c.vol.data = sh.sdf;
            for (int a = 0; a < 3; ++a) {
                c.vol.res[a] = sh.res[a];
                c.vol.origin[a] = sh.sdf_origin[a];
            }
            c.vol.inv_h = 1.0f / sh.sdf_h;
            double far2 = 0.0;  // the lattice corner farthest from the origin
            for (int a = 0; a < 3; ++a) {
                const double lo = sh.sdf_origin[a], hi = lo + (double)sh.sdf_h * (sh.res[a] - 1);
                far2 += std::max(lo * lo, hi * hi);
            }
            reach = std::sqrt(far2);
        } else if (sh.type == MPM_BOX) {
            reach = std::sqrt((double)sh.half[0] * sh.half[0] + (double)sh.half[1] * sh.half[1] +
                              (double)sh.half[2] * sh.half[2]);
        } else {
            reach = (double)sh.half[0] + sh.half[1];
        }
        reach = reach * (1.0 + 1e-4) + 1e-6;  // FP32 rounding of the distance test stays on the safe side
        c.reach2 = (float)(reach * reach);
        float qn = 0.0f;
        for (int a = 0; a < 3; ++a) {
            c.pos[a] = pose[i * 7 + a];
            c.lin[a] = lin_vel[i * 3 + a];
            c.ang[a] = ang_vel ? ang_vel[i * 3 + a] : 0.0f;
            c.com[a] = com ? com[i * 3 + a] : c.pos[a];
        }
        for (int a = 0; a < 4; ++a) {
            c.quat[a] = pose[i * 7 + 3 + a];
            qn += c.quat[a] * c.quat[a];
        }
        if (!(qn > 0.0f) || !std::isfinite(qn)) return MPM_ERR_INVALID_ARG;
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(c.pos[a]) || !std::isfinite(c.lin[a]) || !std::isfinite(c.ang[a]) ||
                !std::isfinite(c.com[a]))
                return MPM_ERR_INVALID_ARG;
    }
    // the device table is only read by work enqueued after this upload, so it is overwritten in place
    ColliderSet* table = s->at<ColliderSet>(s->L.colliders);
    if (k <= kSharedPoses) {  // few bodies: in the kernel parameters, posed per CTA each substep
        ColliderUpload u{};
        u.k = k;
        for (int i = 0; i < k; ++i) u.c[i] = s->stage[i];
        MPM_TRY(launch(s, MPM_K_COLLIDERS, st, [&] {
            return launch_set_colliders_small(u, table, s->at<double>(s->L.wrench), s->substep_counter(), st);
        }, "set_colliders"));
        s->last_upload = u;  // replayed if a pending surrogate step is redone after this upload
    } else {
        MPM_CUDA(cudaMemcpyAsync(table, s->stage, sizeof(ColliderSet) * k, cudaMemcpyHostToDevice, st),
                 "copy colliders");
        MPM_CUDA(cudaEventRecord(s->stage_done, st), "cudaEventRecord");
        MPM_TRY(launch(s, MPM_K_COLLIDERS, st, [&] {
            return launch_set_colliders(table, k, s->at<ColliderNow>(s->L.poses), s->at<double>(s->L.wrench),
                                        s->substep_counter(), s->cfg.dt, st);
        }, "set_colliders"));
    }
    bool changed = s->ncol != k;
    for (int e = 0; e < s->nenv; ++e) {
        const int want = e < (int)s->shape_counts.size() ? s->shape_counts[e] : 0;
        if (s->envs[e].col_count != want) changed = true;
        s->envs[e].col_count = want;
    }
    if (changed) MPM_TRY(upload_envs(s, st));
    s->ncol = k;
    s->upload_seq += 1;
    return MPM_OK;
}

mpm_status mpm_substep(mpm_sim* s, int n_substeps, void* stream) {
    if (!s || n_substeps < 0 || s->sur_pending) return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_substeps == 0) return MPM_OK;
    if (s->N == 0) {
        return launch(s, MPM_K_COLLIDERS, st,
                      [&] { return launch_advance_counter(s->substep_counter(), n_substeps, st); }, "advance");
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MPM_CUDA(cudaStreamIsCapturing(st, &cs), "cudaStreamIsCapturing");
    if (!s->use_graphs || cs != cudaStreamCaptureStatusNone) return enqueue_substeps(s, n_substeps, st);
    GraphEntry* ge = find_graph(s, n_substeps);
    if (!ge) {
        if ((int)s->graphs.size() >= kMaxGraphs) {
            size_t victim = 0;
            for (size_t i = 1; i < s->graphs.size(); ++i)
                if (s->graphs[i].last_use < s->graphs[victim].last_use) victim = i;
            cudaGraphExecDestroy(s->graphs[victim].exec);
            cudaGraphDestroy(s->graphs[victim].graph);
            s->graphs.erase(s->graphs.begin() + victim);
        }
        GraphEntry fresh{};
        MPM_TRY(capture_graph(s, n_substeps, fresh));
        s->graphs.push_back(fresh);
        ge = &s->graphs.back();
    }
    ge->last_use = ++s->use_clock;
    for (auto& tn : ge->timed) {
        cudaEvent_t a = s->get_event(), b = s->get_event();
        MPM_CUDA(cudaGraphExecEventRecordNodeSetEvent(ge->exec, tn.start, a), "cudaGraphExecEventRecordNodeSetEvent");
        MPM_CUDA(cudaGraphExecEventRecordNodeSetEvent(ge->exec, tn.stop, b), "cudaGraphExecEventRecordNodeSetEvent");
        s->pending.push_back({a, b, tn.kind});
    }
    MPM_CUDA(cudaGraphLaunch(ge->exec, st), "cudaGraphLaunch");
    s->ps = ge->after;
    s->launches += ge->launches;
    return MPM_OK;
}

mpm_status mpm_set_graphs(mpm_sim* s, int enable) {
    if (!s) return MPM_ERR_INVALID_ARG;
    s->use_graphs = enable != 0;
    if (!s->use_graphs) s->drop_graphs();
    return MPM_OK;
}

mpm_status mpm_set_launch(mpm_sim* s, int chunk, int fused_ctas_per_sm, int grid_ctas_per_sm) {
    if (!s) return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    if (chunk && (chunk < 32 || chunk > kChunk || chunk % 32)) return MPM_ERR_INVALID_ARG;
    if (grid_ctas_per_sm && (grid_ctas_per_sm < 1 || grid_ctas_per_sm > 8)) return MPM_ERR_INVALID_ARG;
    // the fused pass's CTA size follows the chunk, and its occupancy limit follows the CTA size
    const int new_chunk = chunk ? chunk : s->chunk;
    const bool pen = s->contact == MPM_CONTACT_PARTICLE;
    const int max_fused = transfer_ctas_per_sm(true, s->kind_all, s->nenv == 1, pen, new_chunk);
    if (fused_ctas_per_sm && (fused_ctas_per_sm < 1 || fused_ctas_per_sm > max_fused)) return MPM_ERR_INVALID_ARG;
    // a chunk list cut for another size must be recut before the fused pass runs with this one (its
    // CTA may be smaller than the listed chunks)
    if (new_chunk != s->chunk && s->ps.scanned) s->ps.rechunk = true;
    if (fused_ctas_per_sm)
        s->fused_cps = fused_ctas_per_sm;
    else if (fused_cta_threads(new_chunk) != fused_cta_threads(s->chunk))
        s->fused_cps = max_fused;  // a new CTA size starts at its own occupancy
    else
        s->fused_cps = std::min(s->fused_cps, max_fused);
    s->chunk = new_chunk;
    s->max_fused_cps = max_fused;
    if (grid_ctas_per_sm) s->grid_cps = grid_ctas_per_sm;
    s->drop_graphs();
    return MPM_OK;
}

mpm_status mpm_render_sim(mpm_sim* s, const mpm_camera* cam, const mpm_render_params* params, float* d_depth,
                          float* d_smooth, float* d_normal, float* d_rgb, void* d_workspace, size_t bytes,
                          void* stream) {
    if (!s || !render_args_valid(cam, params)) return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    const StateView v = s->view(s->ps.cur);  // positions in sorted order: the image does not depend on it
    return render_enqueue(*cam, *params, s->N, s->N, v.x, d_depth, d_smooth, d_normal, d_rgb, d_workspace, bytes,
                          static_cast<cudaStream_t>(stream));
}

mpm_status mpm_set_contact(mpm_sim* s, int mode, float stiffness, float damping) {
    if (!s || (mode != MPM_CONTACT_GRID && mode != MPM_CONTACT_PARTICLE)) return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    if (s->net_attached || s->sur_pending) return MPM_ERR_INVALID_ARG;
    if (mode == MPM_CONTACT_PARTICLE) {
        const double dt = s->cfg.dt;
        if (!(stiffness >= 0.0f) || !std::isfinite(stiffness) || (double)stiffness * dt * dt > 1.0) return MPM_ERR_INVALID_ARG;
        if (!(damping >= 0.0f) || !std::isfinite(damping) || (double)damping * dt > 1.0) return MPM_ERR_INVALID_ARG;
    }
    s->contact = mode;
    s->stiffness = mode == MPM_CONTACT_PARTICLE ? stiffness : 0.0f;
    s->damping = mode == MPM_CONTACT_PARTICLE ? damping : 0.0f;
    s->max_fused_cps = transfer_ctas_per_sm(true, s->kind_all, s->nenv == 1, mode == MPM_CONTACT_PARTICLE, s->chunk);
    s->fused_cps = std::min(s->fused_cps, s->max_fused_cps);
    s->drop_graphs();
    return MPM_OK;
}

mpm_status mpm_get_launch(const mpm_sim* s, int* chunk, int* fused_ctas_per_sm, int* grid_ctas_per_sm) {
    if (!s) return MPM_ERR_INVALID_ARG;
    if (chunk) *chunk = s->chunk;
    if (fused_ctas_per_sm) *fused_ctas_per_sm = s->fused_cps;
    if (grid_ctas_per_sm) *grid_ctas_per_sm = s->grid_cps;
    return MPM_OK;
}

// Page-locked host memory (a destination the device copies into without the host waiting).
static bool page_locked(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // (not a pointer the runtime knows: clear the error)
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

mpm_status mpm_read_state(mpm_sim* s, float* x, float* v, float* C, float* F, int dst_on_device, void* stream) {
    if (!s || dst_on_device < 0 || dst_on_device > 2) return MPM_ERR_INVALID_ARG;
    if (dst_on_device == 2)
        for (const float* d : {x, v, C, F})
            if (d && !page_locked(d)) return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (s->N == 0) return MPM_OK;
    const size_t N = (size_t)s->N;
    StateView src = s->view(s->ps.cur);
    if (dst_on_device == 1) {
        return launch(s, MPM_K_READ, st, [&] {
            return launch_read_state(s->N, s->envs_dev(), s->nenv, src, x, v, C, F, st);
        }, "read_state");
    }
    StateView stage = s->view(1 - s->ps.cur);
    MPM_TRY(launch(s, MPM_K_READ, st, [&] {
        return launch_read_state(s->N, s->envs_dev(), s->nenv, src, x ? stage.x : nullptr, v ? stage.v : nullptr,
                                 C ? stage.C : nullptr, F ? stage.F : nullptr, st);
    }, "read_state"));
    if (x) MPM_CUDA(cudaMemcpyAsync(x, stage.x, 3 * N * 4, cudaMemcpyDeviceToHost, st), "copy x");
    if (v) MPM_CUDA(cudaMemcpyAsync(v, stage.v, 3 * N * 4, cudaMemcpyDeviceToHost, st), "copy v");
    if (C) MPM_CUDA(cudaMemcpyAsync(C, stage.C, 9 * N * 4, cudaMemcpyDeviceToHost, st), "copy C");
    if (F) MPM_CUDA(cudaMemcpyAsync(F, stage.F, 9 * N * 4, cudaMemcpyDeviceToHost, st), "copy F");
    // (page-locked destinations: the copies finish in stream order, before the next launch reuses the
    // staging buffer)
    if (dst_on_device == 0) MPM_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return MPM_OK;
}

mpm_status mpm_read_wrench(mpm_sim* s, double* out, int* n_substeps, void* stream) {
    if (!s || (s->ncol > 0 && !out)) return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (s->ncol > 0)
        MPM_CUDA(cudaMemcpyAsync(out, s->at<double>(s->L.wrench), s->ncol * 6 * sizeof(double), cudaMemcpyDeviceToHost,
                                 st),
                 "copy wrench");
    uint32_t cnt = 0;
    MPM_CUDA(cudaMemcpyAsync(&cnt, s->substep_counter(), 4, cudaMemcpyDeviceToHost, st), "copy counter");
    MPM_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (n_substeps) *n_substeps = (int)cnt;
    return MPM_OK;
}

mpm_status mpm_read_wrench_async(mpm_sim* s, double* out, unsigned* n_substeps, void* stream) {
    if (!s || (s->ncol > 0 && (!out || !page_locked(out))) || (n_substeps && !page_locked(n_substeps)))
        return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (s->ncol > 0)
        MPM_CUDA(cudaMemcpyAsync(out, s->at<double>(s->L.wrench), s->ncol * 6 * sizeof(double), cudaMemcpyDeviceToHost,
                                 st),
                 "copy wrench");
    if (n_substeps)
        MPM_CUDA(cudaMemcpyAsync(n_substeps, s->substep_counter(), 4, cudaMemcpyDeviceToHost, st), "copy counter");
    return MPM_OK;
}

mpm_status mpm_get_status(mpm_sim* s, unsigned* flags, int clear, void* stream) {
    if (!s || !flags) return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint32_t f = 0;
    MPM_CUDA(cudaMemcpyAsync(&f, s->status(), 4, cudaMemcpyDeviceToHost, st), "copy status");
    if (clear) MPM_CUDA(cudaMemsetAsync(s->status(), 0, 4, st), "clear status");
    MPM_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    *flags = f;
    return MPM_OK;
}

mpm_status mpm_read_grid(mpm_sim* s, float* d_out, void* stream) {
    if (!s || !d_out) return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (s->N > 0) MPM_TRY(ensure_grid(s, st));
    const float4* grid = s->at<float4>(s->L.grid[s->ps.g]);
    size_t off = 0;
    for (int e = 0; e < s->nenv; ++e) {
        const EnvDesc& d = s->envs[e];
        MPM_TRY(launch(s, MPM_K_READ, st, [&] { return launch_read_grid(d.geo, grid + d.node_base, d_out + off, st); },
                       "read_grid"));
        off += (size_t)d.geo.n * d.geo.n * d.geo.n * 4;
    }
    return MPM_OK;
}

static mpm_box box_from_bins(const int b[6], int margin, int n) {
    if (b[3] < 0) return mpm_box{0, 0, 0, 0, 0, 0};  // no active bins
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = std::max(0, 4 * b[a] - margin);
        hi[a] = std::min(n, 4 * b[3 + a] + 4 + margin);
    }
    return mpm_box{lo[0], lo[1], lo[2], hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
}

mpm_status mpm_surrogate_box(mpm_sim* s, int margin, mpm_box* box, void* stream) {
    if (!s || !box || margin < 0 || s->nenv != 1 || s->sur_pending || s->contact != MPM_CONTACT_GRID)
        return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    *box = mpm_box{0, 0, 0, 0, 0, 0};
    if (s->N == 0) return MPM_OK;
    MPM_TRY(ensure_grid(s, st));
    int* d_box = s->sur_box();
    const Geometry& g = s->envs[0].geo;
    MPM_CUDA(launch_sur_box(s->list(s->ps.g), s->list_count(s->ps.g), g.nb, (int)s->T.bins, d_box, st), "sur_box");
    int b[6];
    MPM_CUDA(cudaMemcpyAsync(b, d_box, sizeof(b), cudaMemcpyDeviceToHost, st), "copy box");
    MPM_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    *box = box_from_bins(b, margin, g.n);
    return MPM_OK;
}

static bool valid_box(const mpm_box* b) {
    return b && b->D > 0 && b->H > 0 && b->W > 0 && (size_t)b->D * b->H * b->W < ((size_t)1 << 31);
}

static SurBox to_sur_box(const mpm_box* b) { return SurBox{b->i0, b->j0, b->k0, b->D, b->H, b->W}; }

mpm_status mpm_surrogate_features(mpm_sim* s, const mpm_box* box, float m_scale, float v_scale, float* d_feat,
                                  uint8_t* d_mask, void* stream) {
    if (!s || s->nenv != 1 || s->sur_pending || !valid_box(box) || !d_feat || !d_mask || s->N == 0)
        return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    if (reinterpret_cast<uintptr_t>(d_feat) % 16) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MPM_TRY(ensure_scanned(s, st));
    MPM_TRY(ensure_grid(s, st));
    double* sums = s->sur_sums();
    MPM_CUDA(cudaMemsetAsync(sums, 0, 16 * sizeof(double), st), "cudaMemsetAsync");
    MPM_CUDA(launch_sur_moments(s->at<float4>(s->L.grid[s->ps.g]), s->list(s->ps.g), s->list_count(s->ps.g),
                                (int)s->T.bins, sums, st),
             "sur_moments");
    if (s->ncol > 0)
        MPM_CUDA(cudaMemcpyAsync(s->sur_wrench(), s->at<double>(s->L.wrench), s->ncol * 6 * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st),
                 "copy wrench");
    MPM_TRY(enqueue_grid_half(s, st));
    const Geometry& g = s->envs[0].geo;
    MPM_CUDA(launch_sur_features(s->at<float4>(s->L.grid[s->ps.g]), g.n, g.nb, to_sur_box(box), m_scale, v_scale,
                                 d_feat, d_mask, sums + 4, st),
             "sur_features");
    s->sur_pending = true;
    return MPM_OK;
}

mpm_status mpm_surrogate_check(mpm_sim* s, const mpm_box* box, const float* d_dv, float dv_unit, int k,
                               double v_ref, double* out, void* stream) {
    if (!s || !s->sur_pending || !valid_box(box) || !d_dv || !out || k < 1 || !(v_ref >= 0.0))
        return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* sums = s->sur_sums();
    MPM_CUDA(cudaMemsetAsync(sums + 7, 0, 3 * sizeof(double), st), "cudaMemsetAsync");
    const Geometry& g = s->envs[0].geo;
    MPM_CUDA(launch_sur_correct(s->at<float4>(s->L.grid[s->ps.g]), g.n, g.nb, s->cfg.bound, to_sur_box(box), d_dv,
                                dv_unit, 0, sums + 7, st),
             "sur_check");
    double h[kSumWindow];
    MPM_CUDA(cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st), "copy sums");
    MPM_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    const double M = h[0];
    const double Mp = (double)s->envs[0].part_count * s->envs[0].mat.p_mass;
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double pexp = h[1 + a] + 0.5 * (k + 1) * (h[4 + a] - h[1 + a]);
        d2 += (h[7 + a] - pexp) * (h[7 + a] - pexp);
    }
    if (v_ref == 0.0) v_ref = M > 0.0 && h[kSumK0] > 0.0 ? std::sqrt(h[kSumK0] / M) : 1e-30;  // the scene's
    out[0] = Mp > 0.0 ? std::fabs(M - Mp) / Mp : 0.0;
    out[1] = M > 0.0 ? std::sqrt(d2) / (M * v_ref) : 0.0;
    out[2] = M;
    out[3] = std::sqrt(d2);
    return MPM_OK;
}

mpm_status mpm_surrogate_advance(mpm_sim* s, const mpm_box* box, const float* d_dv, float dv_unit, int k,
                                 void* stream) {
    if (!s || !s->sur_pending || k < 1 || (d_dv && !valid_box(box))) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s->sur_pending = false;
    if (d_dv) {
        const Geometry& g = s->envs[0].geo;
        MPM_CUDA(launch_sur_correct(s->at<float4>(s->L.grid[s->ps.g]), g.n, g.nb, s->cfg.bound, to_sur_box(box),
                                    d_dv, dv_unit, 1, s->sur_sums() + 12, st),
                 "sur_apply");
        MPM_TRY(enqueue_particle_half(s, st, (float)k * s->cfg.dt));
        if (k > 1) {
            MPM_TRY(launch(s, MPM_K_COLLIDERS, st,
                           [&] { return launch_advance_counter(s->substep_counter(), k - 1, st); }, "advance"));
            MPM_CUDA(launch_wrench_extrapolate(s->at<double>(s->L.wrench), s->sur_wrench(), s->ncol * 6,
                                               (double)(k - 1), st),
                     "wrench_extrapolate");
        }
        return MPM_OK;
    }
    MPM_TRY(enqueue_particle_half(s, st));
    return k > 1 ? enqueue_substeps(s, k - 1, st) : MPM_OK;
}

// ---- attached network: the whole surrogate environment step inside the library (graph-replayed)

namespace {

struct NetLayout {
    size_t feat, xbf, act[3], out, mask, dist, snap, wrench, cols, words, slots, total;
};

// Per-step gate: the sums of up to kGateSlots windows wait for one decision (more windows are decided in
// groups of kGateSlots).
constexpr int kGateSlots = 64;

NetLayout net_layout(int max_voxels, int max_particles = 0) {
    NetLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align_up(bytes);
        return o;
    };
    const size_t v = (size_t)std::max(max_voxels, 1);
    L.feat = take(v * 16);
    L.xbf = take(v * 8);
    for (int i = 0; i < 3; ++i) L.act[i] = take(v * 64);
    L.out = take(v * 12);
    L.mask = take(v);
    L.dist = take(v);  // at least one byte per tile
    // the state at the start of a step (x, v, C, F in the caller's order), its body impulses, substep
    // count and the "a window failed" word, for the per-step fallback
    L.snap = take((size_t)std::max(max_particles, 1) * 49 * sizeof(float));  // raw state + caller-order scratch
    L.wrench = take(MPM_MAX_COLLIDERS * 6 * sizeof(double));
    L.cols = take(MPM_MAX_COLLIDERS * sizeof(ColliderSet));
    L.words = take(4 * sizeof(uint32_t));
    L.slots = take(kGateSlots * kSumWindow * sizeof(double));
    L.total = off;
    return L;
}

constexpr int kNetChannels[5] = {4, 32, 32, 32, 3};

// One window (k substeps) from the current pipeline state: plain grid update, network, device-side gate,
// then both branches enqueued, each running only on its side of the gate.
// gate_mode: 0 no gate; 1 the window's sums go to `slot` (10 doubles, zero) for a decision after the step's
// windows, and the surrogate branch always runs; 2 both branches, each running on its side of the gate.
mpm_status enqueue_window(mpm_sim* s, const mpm_box& b, int gate_mode, cudaStream_t st, double* slot = nullptr) {
    const mpm_surrogate_net& net = s->net;
    const int k = net.k;
    const bool gate_on = gate_mode != 0;
    const NetLayout NL = net_layout(s->net_max_voxels, s->env_cfg[0].max_particles);
    char* ws = s->net_ws;
    const SurBox box = to_sur_box(&b);
    const Geometry& g = s->envs[0].geo;
    if (gate_mode == 1 && !slot) return MPM_ERR_INVALID_ARG;
    double* sums = gate_mode == 1 ? slot : s->sur_sums();
    MPM_TRY(ensure_scanned(s, st));
    MPM_TRY(ensure_grid(s, st));
    if (s->ncol > 0)
        MPM_CUDA(cudaMemcpyAsync(s->sur_wrench(), s->at<double>(s->L.wrench), s->ncol * 6 * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st),
                 "copy wrench");
    // with a gate, the grid update also sums the transfer's mass and momentum (the gate's sums are zero:
    // cleared at attach and by every decision)
    MPM_TRY(enqueue_grid_half(s, st, nullptr, 1, gate_on ? sums : nullptr));
    uint8_t* mask = reinterpret_cast<uint8_t*>(ws + NL.mask);
    uint8_t* dist = reinterpret_cast<uint8_t*>(ws + NL.dist);
    float* dv = reinterpret_cast<float*>(ws + NL.out);
    MPM_CUDA(launch_sur_features(s->at<float4>(s->L.grid[s->ps.g]), g.n, g.nb, box, net.m_scale, net.v_scale,
                                 nullptr, mask, gate_on ? sums + 4 : nullptr, st, ws + NL.xbf),
             "sur_features");
    MPM_TRY(mpm_conv3d_tc_tile_dist(b.D, b.H, b.W, mask, dist, st));
    const void* in = ws + NL.xbf;
    for (int i = 0; i < 4; ++i) {
        const bool last = i == 3;
        void* out = last ? static_cast<void*>(dv) : static_cast<void*>(ws + NL.act[i]);
        MPM_TRY(mpm_conv3d_forward_tc(b.D, b.H, b.W, kNetChannels[i], kNetChannels[i + 1], in, net.w_packed[i],
                                      net.bias[i], last ? 0 : 1, last ? 1 : 0, out, dist, 3 - i, st));
        in = out;
    }
    const double mp = (double)s->envs[0].part_count * s->envs[0].mat.p_mass;
    if (gate_mode == 1) {  // per-step gate: the correction and its momentum sum; decided after the windows
        MPM_CUDA(launch_sur_apply(s->at<float4>(s->L.grid[s->ps.g]), g.n, g.nb, s->cfg.bound, box, dv, net.dv_unit,
                                  nullptr, s->substep_counter(), k, s->at<double>(s->L.wrench), s->sur_wrench(),
                                  s->ncol * 6, st, sums + 7),
                 "sur_apply");
        return enqueue_particle_half(s, st, (float)k * s->cfg.dt);
    }
    if (gate_on)
        MPM_CUDA(launch_sur_check_gate(s->at<float4>(s->L.grid[s->ps.g]), g.n, g.nb, s->cfg.bound, box, dv,
                                       net.dv_unit, sums, mp, k, net.v_ref, net.threshold, s->sur_gate(),
                                       s->sur_stats(), nullptr, s->sur_reduce(), st),
                 "sur_check_gate");
    // without per-window branches every window takes the surrogate branch and the plain one is not enqueued
    uint32_t* gate = gate_mode == 2 ? s->sur_gate() : nullptr;
    const PipeState before = s->ps;
    // the surrogate branch: correction (with the counter and impulse bookkeeping), then the k*dt pass
    MPM_CUDA(launch_sur_apply(s->at<float4>(s->L.grid[s->ps.g]), g.n, g.nb, s->cfg.bound, box, dv, net.dv_unit, gate,
                              s->substep_counter(), k, s->at<double>(s->L.wrench), s->sur_wrench(), s->ncol * 6, st),
             "sur_apply");
    MPM_TRY(enqueue_particle_half(s, st, (float)k * s->cfg.dt, gate, 1u));
    const PipeState after = s->ps;
    if (gate_mode != 2) return MPM_OK;
    // the plain branch, from the same state; with k odd it ends in the same buffers
    s->ps = before;
    MPM_TRY(enqueue_particle_half(s, st, 0.0f, gate, 0u));
    for (int it = 1; it < k; ++it) {
        MPM_TRY(enqueue_grid_half(s, st, gate, 0u));
        MPM_TRY(enqueue_particle_half(s, st, 0.0f, gate, 0u));
    }
    if (!(s->ps == after)) return MPM_ERR_INVALID_ARG;
    return MPM_OK;
}

}  // namespace

// The verdict of a gated surrogate step that returned without waiting for it: wait for it now; if a window
// failed the gate, redo the step from its snapshot with plain substeps (then replay a collider upload made
// after the step, which the caller meant for the next one); otherwise keep the next step's box.
static mpm_status resolve_pending(mpm_sim* s) {
    if (!s->verify_pending) return MPM_OK;
    s->verify_pending = false;
    MPM_CUDA(cudaEventSynchronize(s->verify_event), "cudaEventSynchronize");
    cudaStream_t st = s->verify_stream;
    if (!s->verify_host[0]) {
        s->box_cache = box_from_bins(reinterpret_cast<const int*>(s->verify_host + 1), s->net.margin, s->envs[0].geo.n);
        s->box_cache_ps = s->verify_ps;
        s->box_cache_version = s->particles_version;
        s->box_cache_n = s->N;
        s->box_cached = true;
        return MPM_OK;
    }
    const NetLayout NL = net_layout(s->net_max_voxels, s->env_cfg[0].max_particles);
    float* snap = reinterpret_cast<float*>(s->net_ws + NL.snap);
    const size_t N = (size_t)s->N, cap = std::max<size_t>(s->T.particles, 1);
    float* order = snap + cap * 25;  // the snapshot in the caller's order
    StateView sv;
    sv.x = snap;
    sv.v = snap + 3 * N;
    sv.C = snap + 6 * N;
    sv.F = snap + 15 * N;
    sv.pid = reinterpret_cast<uint32_t*>(snap + 24 * cap);
    MPM_CUDA(launch_read_state(s->N, s->envs_dev(), 1, sv, order, order + 3 * N, order + 6 * N, order + 15 * N, st),
             "snapshot order");
    MPM_TRY(mpm_set_particles(s, s->N, order, order + 3 * N, order + 6 * N, order + 15 * N, 1, st));
    if (s->ncol > 0)
        MPM_CUDA(cudaMemcpyAsync(s->at<ColliderSet>(s->L.colliders), s->net_ws + NL.cols, s->ncol * sizeof(ColliderSet),
                                 cudaMemcpyDeviceToDevice, st),
                 "restore colliders");
    uint32_t* words = reinterpret_cast<uint32_t*>(s->net_ws + NL.words);
    MPM_CUDA(launch_sur_step_restore(s->at<double>(s->L.wrench), reinterpret_cast<const double*>(s->net_ws + NL.wrench),
                                     s->ncol * 6, s->substep_counter(), words, st),
             "step_restore");
    MPM_TRY(mpm_substep(s, s->verify_substeps, st));
    s->sur_steps_redone += 1;
    s->sur_windows_redone += s->verify_substeps / s->net.k;
    if (s->upload_seq != s->verify_upload_seq && s->last_upload.k > 0)
        MPM_TRY(launch(s, MPM_K_COLLIDERS, st, [&] {
            return launch_set_colliders_small(s->last_upload, s->at<ColliderSet>(s->L.colliders),
                                              s->at<double>(s->L.wrench), s->substep_counter(), st);
        }, "set_colliders"));
    return MPM_OK;
}

size_t mpm_surrogate_workspace_size(int max_voxels, int max_particles) {
    return max_voxels > 0 && max_particles >= 0 ? net_layout(max_voxels, max_particles).total : 0;
}

mpm_status mpm_surrogate_attach(mpm_sim* s, const mpm_surrogate_net* net, void* d_workspace, size_t bytes,
                                int max_voxels) {
    if (!s || s->nenv != 1 || !s->tail_scan()) return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    if (net && s->contact != MPM_CONTACT_GRID) return MPM_ERR_INVALID_ARG;  // windows use the grid form
    if (!net) {
        s->net_attached = false;
        s->drop_graphs();
        return MPM_OK;
    }
    if (net->k < 1 || net->k % 2 == 0 || net->margin < 0 || !(net->dv_unit > 0.0f) || !(net->v_ref >= 0.0) ||
        max_voxels < 1 || s->env_cfg[0].max_colliders > kSharedPoses)
        return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    if (!s->verify_event) {
        MPM_CUDA(cudaEventCreateWithFlags(&s->verify_event, cudaEventDisableTiming), "cudaEventCreate");
        MPM_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&s->verify_host), 8 * sizeof(uint32_t), cudaHostAllocDefault),
                 "cudaHostAlloc");
    }
    for (int i = 0; i < 4; ++i)
        if (!net->w_packed[i] || reinterpret_cast<uintptr_t>(net->w_packed[i]) % 16) return MPM_ERR_INVALID_ARG;
    if (!d_workspace || reinterpret_cast<uintptr_t>(d_workspace) % kAlign ||
        bytes < net_layout(max_voxels, s->env_cfg[0].max_particles).total)
        return MPM_ERR_WORKSPACE;
    s->net = *net;
    s->net_ws = static_cast<char*>(d_workspace);
    s->net_max_voxels = max_voxels;
    s->net_attached = true;
    s->drop_graphs();
    // the gate's sums and ticket start at zero (each gate leaves them so)
    const NetLayout NL = net_layout(max_voxels, s->env_cfg[0].max_particles);
    MPM_CUDA(cudaMemset(s->sur_sums(), 0, 16 * sizeof(double)), "cudaMemset");
    MPM_CUDA(cudaMemset(s->net_ws + NL.words, 0, 4 * sizeof(uint32_t)), "cudaMemset");
    MPM_CUDA(cudaMemset(s->net_ws + NL.slots, 0, kGateSlots * kSumWindow * sizeof(double)), "cudaMemset");
    return MPM_OK;
}

mpm_status mpm_surrogate_step(mpm_sim* s, int n_substeps, int gate, void* stream) {
    if (!s || !s->net_attached || s->sur_pending || n_substeps < 0 || n_substeps % s->net.k || gate < 0 || gate > 2)
        return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MPM_TRY(resolve_pending(s));
    if (n_substeps == 0) return MPM_OK;
    mpm_box b{};
    if (s->box_cached && s->box_cache_ps == s->ps && s->box_cache_version == s->particles_version &&
        s->box_cache_n == s->N)
        b = s->box_cache;  // computed at the end of the previous step, from this state
    else
        MPM_TRY(mpm_surrogate_box(s, s->net.margin, &b, stream));
    s->box_cached = false;
    if (b.D == 0 || (size_t)b.D * b.H * b.W > (size_t)s->net_max_voxels) return mpm_substep(s, n_substeps, stream);
    const std::array<int, 8> key{b.i0, b.j0, b.k0, b.D, b.H, b.W, n_substeps, gate};
    const NetLayout NL = net_layout(s->net_max_voxels, s->env_cfg[0].max_particles);
    uint32_t* any_failed = reinterpret_cast<uint32_t*>(s->net_ws + NL.words);
    float* snap = reinterpret_cast<float*>(s->net_ws + NL.snap);
    const size_t cap = std::max<size_t>(s->T.particles, 1);
    // the work around the windows, captured with them: one graph launch per step
    auto step_prologue = [&](cudaStream_t cs) -> mpm_status {
        if (gate == 2) MPM_CUDA(cudaMemsetAsync(s->sur_sums(), 0, 16 * sizeof(double), cs), "cudaMemsetAsync");
        if (gate != 1) return MPM_OK;
        // the step's starting point (the raw state buffer), for a plain redo
        MPM_CUDA(cudaMemcpyAsync(snap, s->at<float>(s->L.state[s->ps.cur]), cap * 25 * sizeof(float),
                                 cudaMemcpyDeviceToDevice, cs),
                 "snapshot");
        MPM_CUDA(launch_sur_step_begin(s->at<double>(s->L.wrench), reinterpret_cast<double*>(s->net_ws + NL.wrench),
                                       s->ncol * 6, s->substep_counter(), any_failed, cs),
                 "step_begin");
        if (s->ncol > 0)
            MPM_CUDA(cudaMemcpyAsync(s->net_ws + NL.cols, s->at<ColliderSet>(s->L.colliders),
                                     s->ncol * sizeof(ColliderSet), cudaMemcpyDeviceToDevice, cs),
                     "snapshot colliders");
        return MPM_OK;
    };
    // per-step gate: the verdict and the next step's box, copied to pinned host memory (read lazily)
    auto step_epilogue = [&](cudaStream_t cs) -> mpm_status {
        if (gate != 1) return MPM_OK;
        int* d_box = s->sur_box();
        const Geometry& g = s->envs[0].geo;
        MPM_CUDA(launch_sur_box(s->list(s->ps.g), s->list_count(s->ps.g), g.nb, (int)s->T.bins, d_box, cs), "sur_box");
        MPM_CUDA(cudaMemcpyAsync(s->verify_host, any_failed, sizeof(uint32_t), cudaMemcpyDeviceToHost, cs),
                 "copy flag");
        MPM_CUDA(cudaMemcpyAsync(s->verify_host + 1, d_box, 6 * sizeof(int), cudaMemcpyDeviceToHost, cs), "copy box");
        return MPM_OK;
    };
    GraphEntry* ge = nullptr;
    for (size_t i = 0; i < s->sur_graphs.size(); ++i)
        if (s->sur_keys[i] == key && s->sur_graphs[i].before == s->ps && s->sur_graphs[i].ncol == s->ncol)
            ge = &s->sur_graphs[i];
    if (!ge) {
        if (s->sur_graphs.size() >= 16) {  // keep a bounded cache
            cudaGraphExecDestroy(s->sur_graphs.front().exec);
            cudaGraphDestroy(s->sur_graphs.front().graph);
            s->sur_graphs.erase(s->sur_graphs.begin());
            s->sur_keys.erase(s->sur_keys.begin());
        }
        if (!s->cap_stream)
            MPM_CUDA(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        GraphEntry fresh{};
        fresh.n_substeps = n_substeps;
        fresh.N = s->N;
        fresh.ncol = s->ncol;
        fresh.before = s->ps;
        const long long l0 = s->launches;
        const unsigned mask_saved = s->timing_mask;
        s->timing_mask = 0;  // no timing events inside these graphs
        MPM_CUDA(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        s->capturing = true;
        mpm_status r = step_prologue(s->cap_stream);
        const int nwin = n_substeps / s->net.k;
        double* slots = reinterpret_cast<double*>(s->net_ws + NL.slots);
        const double mp = (double)s->envs[0].part_count * s->envs[0].mat.p_mass;
        for (int w = 0; w < nwin && r == MPM_OK; ++w) {
            r = enqueue_window(s, b, gate, s->cap_stream, slots + (size_t)(w % kGateSlots) * kSumWindow);
            const int done = w % kGateSlots + 1;  // windows waiting in the slots
            if (r == MPM_OK && gate == 1 && (done == kGateSlots || w + 1 == nwin)) {
                const cudaError_t e = launch_sur_decide(slots, done, mp, s->net.k, s->net.v_ref, s->net.threshold,
                                                        s->sur_stats(), any_failed, s->cap_stream);
                if (e != cudaSuccess) r = cuda_fail(e, "sur_decide");
            }
        }
        if (r == MPM_OK) r = step_epilogue(s->cap_stream);
        s->capturing = false;
        s->timing_mask = mask_saved;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(s->cap_stream, &graph);
        fresh.after = s->ps;
        fresh.launches = s->launches - l0;
        s->ps = fresh.before;
        s->launches = l0;
        if (r != MPM_OK) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&fresh.exec, graph, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(graph);
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        fresh.graph = graph;
        s->sur_graphs.push_back(fresh);
        s->sur_keys.push_back(key);
        ge = &s->sur_graphs.back();
    }
    MPM_CUDA(cudaGraphLaunch(ge->exec, st), "cudaGraphLaunch");
    s->ps = ge->after;
    s->launches += ge->launches;
    if (gate == 1) {  // the verdict and the next step's box were copied by the graph; read them lazily
        MPM_CUDA(cudaEventRecord(s->verify_event, st), "cudaEventRecord");
        s->verify_pending = true;
        s->verify_substeps = n_substeps;
        s->verify_stream = st;
        s->verify_ps = s->ps;
        s->verify_upload_seq = s->upload_seq;
    }
    return MPM_OK;
}

mpm_status mpm_surrogate_stats(mpm_sim* s, long long* windows, long long* fallbacks, double* residuals, int reset,
                               void* stream) {
    if (!s) return MPM_ERR_INVALID_ARG;
    MPM_TRY(resolve_pending(s));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long h[4];
    MPM_CUDA(cudaMemcpyAsync(h, s->sur_stats(), sizeof(h), cudaMemcpyDeviceToHost, st), "copy stats");
    if (reset) MPM_CUDA(cudaMemsetAsync(s->sur_stats(), 0, 2 * sizeof(unsigned long long), st), "cudaMemsetAsync");
    MPM_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (windows) *windows = (long long)h[0];
    // per-window branches: the windows that failed the gate; per-step fallback: the windows of redone steps
    if (fallbacks) *fallbacks = (long long)h[1] + s->sur_windows_redone;
    if (reset) s->sur_steps_redone = s->sur_windows_redone = 0;
    if (residuals) std::memcpy(residuals, &h[2], 2 * sizeof(double));
    return MPM_OK;
}

mpm_status mpm_set_timing(mpm_sim* s, unsigned kernel_mask) {
    if (!s) return MPM_ERR_INVALID_ARG;
    s->timing_mask = kernel_mask & ((1u << MPM_K_COUNT) - 1u);
    return MPM_OK;
}

mpm_status mpm_read_timing(mpm_sim* s, double* ms, long long* launches, int reset) {
    if (!s) return MPM_ERR_INVALID_ARG;
    for (auto& ev : s->pending) {
        MPM_CUDA(cudaEventSynchronize(ev.b), "cudaEventSynchronize");
        float t = 0.0f;
        MPM_CUDA(cudaEventElapsedTime(&t, ev.a, ev.b), "cudaEventElapsedTime");
        s->ms[ev.kind] += t;
        s->counts[ev.kind] += 1;
        s->pool.push_back(ev.a);
        s->pool.push_back(ev.b);
    }
    s->pending.clear();
    for (int k = 0; k < MPM_K_COUNT; ++k) {
        if (ms) ms[k] = s->ms[k];
        if (launches) launches[k] = s->counts[k];
    }
    if (reset) {
        for (int k = 0; k < MPM_K_COUNT; ++k) {
            s->ms[k] = 0.0;
            s->counts[k] = 0;
        }
    }
    return MPM_OK;
}

}  // extern "C"
