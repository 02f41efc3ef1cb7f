// mpm_abi.cu -- the C-ABI of include/mpm.h: argument checks, workspace layout, the per-substep launch
// sequence (optionally replayed from a CUDA graph) and the readbacks. All device memory comes from the
// caller's workspace.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "mpm.h"
#include "mpm_internal.h"

using namespace mpm;

namespace {

thread_local char g_last_error[256] = "";

mpm_status cuda_fail(cudaError_t e, const char* what) {
    snprintf(g_last_error, sizeof g_last_error, "%s: %s", what, cudaGetErrorString(e));
    return MPM_ERR_CUDA;
}

#define MPM_CUDA(call, what)                               \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

#define MPM_TRY(call)                   \
    do {                                \
        mpm_status r_ = (call);         \
        if (r_ != MPM_OK) return r_;    \
    } while (0)

constexpr size_t kAlign = 256;
constexpr int kMaxGraphs = 8;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
    size_t state[2], key, perm, grid[2], flags[2], hist, list[2], list_meta, cursor, chunks, colliders, wrench,
        counters, total;
    size_t max_chunks;
};

Layout make_layout(const mpm_config& c) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align_up(bytes);
        return o;
    };
    const size_t Nmax = (size_t)c.max_particles;
    const size_t nb = (size_t)c.n / 4;
    const size_t nblocks = nb * nb * nb;
    const size_t nodes = nblocks * kBlkNodes;
    for (int i = 0; i < 2; ++i) L.state[i] = take(Nmax * 25 * 4);
    L.key = take(Nmax * 8);  // (bin, rank within bin) per particle
    L.perm = take(Nmax * 4);
    for (int i = 0; i < 2; ++i) L.grid[i] = take(nodes * sizeof(float4));
    for (int i = 0; i < 2; ++i) L.flags[i] = take(nblocks * 4);
    L.hist = take(nblocks * 4);
    for (int i = 0; i < 2; ++i) L.list[i] = take(nblocks * 4);
    L.list_meta = take(4 * sizeof(uint32_t));  // list counts [2], grid-update CTAs done, spare
    // everything from grid[0] up to here restarts from zero on mpm_set_particles
    L.cursor = take(nblocks * 4);
    L.max_chunks = Nmax / kChunk + nblocks + 1;
    L.chunks = take(L.max_chunks * sizeof(int4));
    L.colliders = take(kMaxColliders * sizeof(ColliderSet));
    L.wrench = take(kMaxColliders * 6 * sizeof(double));
    L.counters = take(4 * sizeof(uint32_t));  // status, substep counter, num_chunks, CTAs done
    L.total = off;
    return L;
}

mpm_status check_config(const mpm_config* c, const mpm_material* m) {
    if (!c || !m) return MPM_ERR_INVALID_ARG;
    if (c->n < 8 || c->n > 256 || (c->n % 4) != 0) return MPM_ERR_INVALID_ARG;
    if (!(c->dt > 0.0f) || !std::isfinite(c->dt)) return MPM_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(c->gravity[a])) return MPM_ERR_INVALID_ARG;
    if (c->bound < 0 || 2 * c->bound > c->n) return MPM_ERR_INVALID_ARG;
    if (c->max_particles < 1 || c->max_particles > (1 << 30)) return MPM_ERR_INVALID_ARG;
    if (c->max_colliders < 0 || c->max_colliders > MPM_MAX_COLLIDERS) return MPM_ERR_INVALID_ARG;
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

// Host-side pipeline state that the enqueued work depends on (and that a cached graph assumes).
struct PipeState {
    int cur = 0;               // state buffer holding the current particles
    int g = 0;                 // grid holding the particle-to-grid transfer of the current state
    bool scanned = false;      // bin offsets and chunk list match the current keys
    bool order_valid = false;  // perm (sorted slot -> particle) matches them too
    bool grid_valid = false;   // grid g holds the transfer of the current state
    bool operator==(const PipeState& o) const {
        return cur == o.cur && g == o.g && scanned == o.scanned && order_valid == o.order_valid &&
               grid_valid == o.grid_valid;
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
    mpm_material mat;
    Layout L;
    char* ws;
    Geometry geo;
    Material dmat;
    int N = 0;
    PipeState ps;
    int nshapes = 0;
    mpm_shape shapes[MPM_MAX_COLLIDERS];
    int ncol = 0;  // colliders uploaded by the last mpm_set_colliders
    int sms = 0;
    int ctas_fused = 0, ctas_p2g = 0, ctas_grid = 0;
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
    uint32_t* list(int which) { return at<uint32_t>(L.list[which]); }
    uint32_t* list_count(int which) { return at<uint32_t>(L.list_meta) + which; }
    uint32_t* grid_done() { return at<uint32_t>(L.list_meta) + 2; }
    StateView view(int which) {
        float* b = at<float>(L.state[which]);
        const size_t n = (size_t)N;
        StateView s;
        s.x = b;
        s.v = b + 3 * n;
        s.C = b + 6 * n;
        s.F = b + 15 * n;
        s.pid = reinterpret_cast<uint32_t*>(b + 24 * (size_t)cfg.max_particles);
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
        for (auto& ge : graphs) {
            cudaGraphExecDestroy(ge.exec);
            cudaGraphDestroy(ge.graph);
        }
        graphs.clear();
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

TransferParams transfer_params(mpm_sim* s) {
    TransferParams p{};
    p.geo = s->geo;
    p.mat = s->dmat;
    p.N = s->N;
    p.in = s->view(s->ps.cur);
    p.out = s->view(1 - s->ps.cur);
    p.perm = s->at<uint32_t>(s->L.perm);
    p.keyrank_out = s->at<uint2>(s->L.key);
    p.hist = s->at<uint32_t>(s->L.hist);
    p.chunks = s->at<int4>(s->L.chunks);
    p.num_chunks = s->num_chunks();
    p.status = s->status();
    p.substep_counter = s->substep_counter();
    p.cursor = s->at<uint32_t>(s->L.cursor);
    p.chunks_next = s->at<int4>(s->L.chunks);
    p.num_chunks_next = s->num_chunks();
    p.done = s->done();
    return p;
}

GridParams grid_params(mpm_sim* s) {
    GridParams gp{};
    gp.geo = s->geo;
    for (int a = 0; a < 3; ++a) gp.gravity[a] = s->cfg.gravity[a];
    gp.bound = s->cfg.bound;
    gp.grid = s->at<float4>(s->L.grid[s->ps.g]);
    gp.list = s->list(s->ps.g);
    gp.list_count = s->list_count(s->ps.g);
    gp.list_old = s->list(1 - s->ps.g);
    gp.list_count_old = s->list_count(1 - s->ps.g);
    gp.done = s->grid_done();
    gp.grid_old = s->at<float4>(s->L.grid[1 - s->ps.g]);
    gp.flags_old = s->at<uint32_t>(s->L.flags[1 - s->ps.g]);
    gp.cols = s->at<ColliderSet>(s->L.colliders);
    gp.ncol = s->ncol;
    gp.substep_counter = s->substep_counter();
    gp.ctas = s->ctas_grid;
    gp.wrench = s->at<double>(s->L.wrench);
    return gp;
}

mpm_status ensure_scanned(mpm_sim* s, cudaStream_t st) {
    if (s->ps.scanned) return MPM_OK;
    MPM_TRY(launch(s, MPM_K_SCAN, st, [&] {
        return launch_scan(s->at<uint32_t>(s->L.hist), s->at<uint32_t>(s->L.cursor), s->at<int4>(s->L.chunks),
                           s->num_chunks(), s->geo.nblocks, kChunk, st);
    }, "scan"));
    s->ps.scanned = true;
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
    MPM_TRY(launch(s, MPM_K_P2G, st, [&] { return launch_p2g(p, s->mat.kind, s->ctas_p2g, kChunk, st); }, "p2g"));
    s->ps.grid_valid = true;
    return MPM_OK;
}

// The launches of n substeps: per substep one sort-assign + grid-update launch and one fused
// G2P->P2G launch (whose last CTA sorts the new positions into bins).
mpm_status enqueue_substeps(mpm_sim* s, int n, cudaStream_t st) {
    for (int it = 0; it < n; ++it) {
        MPM_TRY(ensure_scanned(s, st));
        MPM_TRY(ensure_grid(s, st));
        AssignGridParams ap{};
        ap.grid = grid_params(s);
        ap.N = s->N;
        ap.keyrank = s->at<uint2>(s->L.key);
        ap.cursor = s->at<uint32_t>(s->L.cursor);
        ap.perm = s->at<uint32_t>(s->L.perm);
        ap.assign_ctas = s->ps.order_valid ? 0 : (s->N + 1023) / 1024;  // 4 particles per thread
        MPM_TRY(launch(s, MPM_K_GRID, st, [&] { return launch_assign_grid(ap, st); }, "assign_grid"));
        s->ps.order_valid = true;
        TransferParams p = transfer_params(s);
        p.grid_in = ap.grid.grid;
        p.grid_out = ap.grid.grid_old;
        p.flags_out = ap.grid.flags_old;
        p.list_out = s->list(1 - s->ps.g);
        p.list_count_out = s->list_count(1 - s->ps.g);
        MPM_TRY(launch(s, MPM_K_G2P2G, st, [&] { return launch_g2p2g(p, s->mat.kind, s->ctas_fused, kChunk, st); },
                       "g2p2g"));
        s->ps.cur = 1 - s->ps.cur;
        s->ps.g = 1 - s->ps.g;
        s->ps.scanned = true;       // the fused pass's last CTA wrote the new bins
        s->ps.order_valid = false;  // assigned by the next launch
        s->ps.grid_valid = true;
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

}  // namespace

extern "C" {

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

mpm_status mpm_workspace_size(const mpm_config* cfg, const mpm_material* mat, size_t* bytes) {
    if (!bytes) return MPM_ERR_INVALID_ARG;
    MPM_TRY(check_config(cfg, mat));
    *bytes = make_layout(*cfg).total;
    return MPM_OK;
}

mpm_status mpm_create(const mpm_config* cfg, const mpm_material* mat, void* d_workspace, size_t bytes, void* stream,
                      mpm_sim** out) {
    if (!out) return MPM_ERR_INVALID_ARG;
    *out = nullptr;
    MPM_TRY(check_config(cfg, mat));
    Layout L = make_layout(*cfg);
    if (!d_workspace || (reinterpret_cast<uintptr_t>(d_workspace) % kAlign) != 0 || bytes < L.total)
        return MPM_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    mpm_sim* s = new (std::nothrow) mpm_sim();
    if (!s) return MPM_ERR_INVALID_ARG;
    s->cfg = *cfg;
    s->mat = *mat;
    s->L = L;
    s->ws = static_cast<char*>(d_workspace);
    Geometry& g = s->geo;
    g.n = cfg->n;
    g.nb = cfg->n / 4;
    g.nblocks = g.nb * g.nb * g.nb;
    g.dx = (float)(1.0 / cfg->n);
    g.inv_dx = (float)cfg->n;
    g.dt = cfg->dt;
    g.lo = (float)(2.0 / cfg->n);
    g.hi = (float)(1.0 - 2.0 / cfg->n);
    double mu, lambda;
    if (mat->kind == MPM_PLASTICINE) {
        mu = (double)mat->E / (2.0 * (1.0 + mat->nu));
        lambda = (double)mat->E * mat->nu / ((1.0 + mat->nu) * (1.0 - 2.0 * mat->nu));
    } else {
        mu = 0.0;
        lambda = mat->bulk_modulus;
    }
    s->dmat.mu = (float)mu;
    s->dmat.lambda = (float)lambda;
    s->dmat.yield_radius = mu > 0.0 ? (float)(mat->yield_stress / (2.0 * mu)) : 0.0f;
    s->dmat.p_mass = (float)((double)mat->rho * mat->p_vol);
    s->dmat.stress_scale = (float)(-(double)cfg->dt * mat->p_vol * 4.0 * cfg->n * cfg->n);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "device query");
    }
    s->ctas_fused = s->sms * transfer_ctas_per_sm(mat->kind, kChunk, true);
    s->ctas_p2g = s->sms * transfer_ctas_per_sm(mat->kind, kChunk, false);
    // persistent grid update: two CTAs per SM, or one per group of four bins if that is fewer
    s->ctas_grid = std::min(2 * s->sms, (g.nblocks + 3) / 4);
    // zero the grids, bin flags and counts, colliders and counters
    const size_t zero_from = L.grid[0];
    e = cudaMemsetAsync(s->ws + zero_from, 0, L.total - zero_from, st);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "cudaMemsetAsync");
    }
    *out = s;
    return MPM_OK;
}

void mpm_destroy(mpm_sim* s) {
    if (!s) return;
    s->drop_graphs();
    for (auto& ev : s->pending) {
        cudaEventDestroy(ev.a);
        cudaEventDestroy(ev.b);
    }
    for (auto e : s->pool) cudaEventDestroy(e);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    delete s;
}

int mpm_num_particles(const mpm_sim* s) { return s ? s->N : 0; }

long long mpm_launch_count(const mpm_sim* s) { return s ? s->launches : 0; }

mpm_status mpm_set_particles(mpm_sim* s, int n, const float* x, const float* v, const float* C, const float* F,
                             int src_on_device, void* stream) {
    if (!s || n < 0 || (n > 0 && !x)) return MPM_ERR_INVALID_ARG;
    if (n > s->cfg.max_particles) return MPM_ERR_CAPACITY;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // grids, bin flags and histogram restart from zero
    const size_t z0 = s->L.grid[0], z1 = s->L.cursor;
    MPM_CUDA(cudaMemsetAsync(s->ws + z0, 0, z1 - z0, st), "cudaMemsetAsync");
    s->N = n;
    s->ps = PipeState{};
    if (n == 0) {
        s->ps.scanned = s->ps.order_valid = s->ps.grid_valid = true;
        return MPM_OK;
    }
    const size_t N = (size_t)n;
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
    StateView dst = s->view(0);
    MPM_TRY(launch(s, MPM_K_LOAD, st, [&] {
        return launch_load(s->geo, s->mat.kind, n, sx, sv, sC, sF, dst, s->at<uint2>(s->L.key),
                           s->at<uint32_t>(s->L.hist), s->status(), st);
    }, "load"));
    if (!src_on_device) MPM_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return MPM_OK;
}

mpm_status mpm_set_shapes(mpm_sim* s, int k, const mpm_shape* shapes) {
    if (!s || k < 0 || (k > 0 && !shapes)) return MPM_ERR_INVALID_ARG;
    if (k > s->cfg.max_colliders) return MPM_ERR_CAPACITY;
    for (int i = 0; i < k; ++i) {
        const mpm_shape& sh = shapes[i];
        if (sh.type != MPM_BOX && sh.type != MPM_CAPSULE) return MPM_ERR_INVALID_ARG;
        if (!(sh.friction >= 0.0f) || !std::isfinite(sh.friction)) return MPM_ERR_INVALID_ARG;
        int dims = sh.type == MPM_BOX ? 3 : 2;
        for (int a = 0; a < dims; ++a)
            if (!(sh.half[a] >= 0.0f) || !std::isfinite(sh.half[a])) return MPM_ERR_INVALID_ARG;
    }
    s->nshapes = k;
    if (k) memcpy(s->shapes, shapes, sizeof(mpm_shape) * k);
    return MPM_OK;
}

mpm_status mpm_set_colliders(mpm_sim* s, int k, const float* pose, const float* lin_vel, const float* ang_vel,
                             const float* com, void* stream) {
    if (!s || k != s->nshapes || (k > 0 && (!pose || !lin_vel))) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ColliderUpload u{};
    u.k = k;
    for (int i = 0; i < k; ++i) {
        ColliderSet& c = u.c[i];
        const mpm_shape& sh = s->shapes[i];
        c.type = sh.type;
        for (int a = 0; a < 3; ++a) c.half[a] = sh.half[a];
        c.friction = sh.friction;
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
    MPM_TRY(launch(s, MPM_K_COLLIDERS, st, [&] {
        return launch_set_colliders(u, s->at<ColliderSet>(s->L.colliders), s->at<double>(s->L.wrench),
                                    s->substep_counter(), st);
    }, "set_colliders"));
    s->ncol = k;
    return MPM_OK;
}

mpm_status mpm_substep(mpm_sim* s, int n_substeps, void* stream) {
    if (!s || n_substeps < 0) return MPM_ERR_INVALID_ARG;
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

mpm_status mpm_read_state(mpm_sim* s, float* x, float* v, float* C, float* F, int dst_on_device, void* stream) {
    if (!s) return MPM_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (s->N == 0) return MPM_OK;
    const size_t N = (size_t)s->N;
    StateView src = s->view(s->ps.cur);
    if (dst_on_device) {
        return launch(s, MPM_K_READ, st, [&] { return launch_read_state(s->mat.kind, s->N, src, x, v, C, F, st); },
                      "read_state");
    }
    StateView stage = s->view(1 - s->ps.cur);
    MPM_TRY(launch(s, MPM_K_READ, st, [&] {
        return launch_read_state(s->mat.kind, s->N, src, x ? stage.x : nullptr, v ? stage.v : nullptr,
                                 C ? stage.C : nullptr, F ? stage.F : nullptr, st);
    }, "read_state"));
    if (x) MPM_CUDA(cudaMemcpyAsync(x, stage.x, 3 * N * 4, cudaMemcpyDeviceToHost, st), "copy x");
    if (v) MPM_CUDA(cudaMemcpyAsync(v, stage.v, 3 * N * 4, cudaMemcpyDeviceToHost, st), "copy v");
    if (C) MPM_CUDA(cudaMemcpyAsync(C, stage.C, 9 * N * 4, cudaMemcpyDeviceToHost, st), "copy C");
    if (F) MPM_CUDA(cudaMemcpyAsync(F, stage.F, 9 * N * 4, cudaMemcpyDeviceToHost, st), "copy F");
    MPM_CUDA(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return MPM_OK;
}

mpm_status mpm_read_wrench(mpm_sim* s, double* out, int* n_substeps, void* stream) {
    if (!s || (s->ncol > 0 && !out)) return MPM_ERR_INVALID_ARG;
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

mpm_status mpm_get_status(mpm_sim* s, unsigned* flags, int clear, void* stream) {
    if (!s || !flags) return MPM_ERR_INVALID_ARG;
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
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (s->N > 0) MPM_TRY(ensure_grid(s, st));
    const float4* grid = s->at<float4>(s->L.grid[s->ps.g]);
    return launch(s, MPM_K_READ, st, [&] { return launch_read_grid(s->geo, grid, d_out, st); }, "read_grid");
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
