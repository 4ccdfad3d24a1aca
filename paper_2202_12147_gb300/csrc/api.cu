// C ABI of liblbib (declared in include/lbib.h): argument checks, the layout
// of the caller buffers, mesh preprocessing, CUDA-graph capture of the step
// and the host-side accessors.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "lbib_internal.cuh"

using namespace lbib;

namespace {

thread_local std::string g_last_error;

}  // namespace

void lbib::set_last_error(const char *msg) { g_last_error = msg; }

namespace {

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

#define CU(call)                                                                               \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(LBIB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));       \
    } while (0)

constexpr size_t ALIGN = 256;
size_t up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

constexpr int GRAPH_STEPS = 16;  // steps per captured graph (even: both AA parities)

int env_int(const char *name, int dflt) {
    const char *v = getenv(name);
    return (v && v[0]) ? atoi(v) : dflt;
}

// Replay the captured CUDA graphs (default) or launch each step's kernels
// directly (LBIB_GRAPHS=0).  The graphs are instantiated with per-node
// priorities, so the immersed-boundary branch keeps its stream's high
// priority inside a replay; without that a replayed step of a 256 x 128 x 128
// two-swimmer box took 131 us, with it 105 us (direct launches: 108 us).
bool use_graphs(long long) { return env_int("LBIB_GRAPHS", 1) != 0; }


struct Layout {
    long long N = 0, Npad = 0;
    int n_tiles = 0, tile_x = 0, tiles_x = 0;
    size_t esize = 4;
    size_t bytes[LBIB_NBUF] = {0, 0, 0};
    // fields
    size_t oF = 0, oFdet = 0, oU = 0, oMarks = 0, oList = 0, oCount = 0;
    // aux
    int n_edges = 0;
    size_t oedge = 0, ovg = 0, ovfix = 0;
    size_t orx = 0, ory = 0, orz = 0, onf = 0, onv = 0, otf = 0, otri = 0, ocp = 0, oce = 0, onb = 0,
           obead = 0, oswim = 0, obd = 0, obe = 0, octl = 0, osws = 0, oxcm = 0, oswp = 0, obv = 0, otrk = 0, obacc = 0;
};

bool valid_params(const lb_params *p, std::string &why) {
    if (!p) { why = "params is NULL"; return false; }
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) { why = "box dimensions must be >= 1"; return false; }
    long long N = (long long)p->nx * p->ny * p->nz;
    if (N >= (1ll << 31)) { why = "box has 2^31 cells or more"; return false; }
    if (!(p->tau > 0.5)) { why = "tau must exceed 1/2 (positive viscosity)"; return false; }
    if (!(p->rho0 > 0.0)) { why = "rho0 must be positive"; return false; }
    if (p->storage < LBIB_F32 || p->storage > LBIB_BF16) { why = "unknown storage format"; return false; }
    if (p->forcing != LBIB_GUO && p->forcing != LBIB_SHAN_CHEN) { why = "unknown forcing scheme"; return false; }
    if (p->kernel != LBIB_PESKIN4 && p->kernel != LBIB_LINEAR2) { why = "unknown delta kernel"; return false; }
    if (p->store_scale < 0.0) { why = "store_scale must be >= 0"; return false; }
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->g[a])) { why = "g must be finite"; return false; }
    return true;
}

// directed edge a -> b of a triangle as one key
inline long long edge_key(int a, int b) { return ((long long)a << 32) | (unsigned)b; }

// third node of the triangle of bead d that runs a -> b along its boundary,
// for every directed edge of the bead's triangles (-1 if two triangles share one)
std::unordered_map<long long, int> directed_edges(const lbib_structure *s, const lbib_bead &d) {
    std::unordered_map<long long, int> m;
    m.reserve(3 * (size_t)d.tri_count);
    for (int t = d.tri_start; t < d.tri_start + d.tri_count; ++t) {
        const int *v = s->tris + 3 * t;
        for (int q = 0; q < 3; ++q) {
            auto r = m.emplace(edge_key(v[q], v[(q + 1) % 3]), v[(q + 2) % 3]);
            if (!r.second) r.first->second = -1;
        }
    }
    return m;
}

bool closed_surface(const lbib_structure *s, const lbib_bead &d) {
    const auto m = directed_edges(s, d);
    for (const auto &kv : m) {
        if (kv.second < 0) return false;
        const int a = (int)(kv.first >> 32), b = (int)(kv.first & 0xffffffffll);
        auto it = m.find(edge_key(b, a));
        if (it == m.end() || it->second < 0) return false;
    }
    return true;
}

// bending edges of one bead in a fixed order (by triangle, then corner): the
// edge a -> b of a triangle (third node c) with a < b, and d the third node of
// the triangle running b -> a
std::vector<std::array<int, 4>> bending_edges(const lbib_structure *s, const lbib_bead &d) {
    const auto m = directed_edges(s, d);
    std::vector<std::array<int, 4>> out;
    for (int t = d.tri_start; t < d.tri_start + d.tri_count; ++t) {
        const int *v = s->tris + 3 * t;
        for (int q = 0; q < 3; ++q) {
            const int a = v[q], b = v[(q + 1) % 3], c = v[(q + 2) % 3];
            if (a < b) out.push_back({a, b, c, m.at(edge_key(b, a))});
        }
    }
    return out;
}

bool valid_structure(const lb_params *p, const lbib_structure *s, std::string &why) {
    if (!s) return true;
    if (s->n_beads < 0 || s->n_swimmers < 0 || s->n_nodes < 0 || s->n_tris < 0) { why = "negative count"; return false; }
    if (s->n_swimmers > 0 && (!s->swimmers || !s->beads)) { why = "swimmer/bead table missing"; return false; }
    if (s->n_nodes > 0 && !s->rest_nodes) { why = "rest_nodes missing"; return false; }
    if (s->n_tris > 0 && !s->tris) { why = "tris missing"; return false; }
    if (s->n_beads != 3 * s->n_swimmers) { why = "every bead must belong to exactly one three-bead swimmer"; return false; }
    std::vector<int> owner(s->n_beads, -1);
    for (int k = 0; k < s->n_swimmers; ++k) {
        const lbib_swimmer &w = s->swimmers[k];
        for (int q = 0; q < 3; ++q) {
            int b = w.bead[q];
            if (b < 0 || b >= s->n_beads) { why = "swimmer bead index out of range"; return false; }
            if (owner[b] >= 0) { why = "bead used by two swimmers"; return false; }
            owner[b] = k;
        }
        if (!(w.period > 0.0) || !std::isfinite(w.k_spring) || !(w.L_spring >= 0.0)) {
            why = "swimmer needs period > 0, finite k_spring, L_spring >= 0";
            return false;
        }
    }
    for (int b = 0; b < s->n_beads; ++b) {
        const lbib_bead &d = s->beads[b];
        if (d.node_count < 4 || d.node_start < 0 || d.node_start + d.node_count > s->n_nodes) {
            why = "bead node range invalid";
            return false;
        }
        if (d.tri_count < 1 || d.tri_start < 0 || d.tri_start + d.tri_count > s->n_tris) {
            why = "bead triangle range invalid";
            return false;
        }
        for (int t = d.tri_start; t < d.tri_start + d.tri_count; ++t)
            for (int q = 0; q < 3; ++q) {
                int v = s->tris[3 * t + q];
                if (v < d.node_start || v >= d.node_start + d.node_count) {
                    why = "triangle uses a node outside its bead";
                    return false;
                }
            }
        if (d.law != LBIB_NEOHOOKE && d.law != LBIB_SKALAK) { why = "unknown membrane law"; return false; }
        if (!std::isfinite(d.Gs) || !std::isfinite(d.C) || !(d.kb >= 0.0) || !(d.kv >= 0.0) || !std::isfinite(d.kb) ||
            !std::isfinite(d.kv)) {
            why = "membrane moduli must be finite, kb and kv >= 0";
            return false;
        }
        if ((d.kb > 0.0 || d.kv > 0.0) && !closed_surface(s, d)) {
            why = "bending and volume terms need a closed surface (every edge on exactly two triangles, "
                  "consistently oriented)";
            return false;
        }
    }
    for (long long j = 0; j < 3ll * s->n_nodes; ++j)
        if (!std::isfinite(s->rest_nodes[j])) { why = "non-finite node coordinate"; return false; }
    (void)p;
    return true;
}

Layout make_layout(const lb_params *p, const lbib_structure *s) {
    Layout L;
    L.N = (long long)p->nx * p->ny * p->nz;
    L.Npad = (L.N + 63) / 64 * 64;
    L.esize = p->storage == LBIB_F32 ? 4 : 2;
    L.tile_x = p->nx <= LB_TPB ? p->nx : LB_TPB;
    L.tiles_x = (p->nx + L.tile_x - 1) / L.tile_x;
    L.n_tiles = L.tiles_x * p->ny * p->nz;
    L.bytes[0] = up((size_t)Q * L.Npad * L.esize);
    size_t o = 0;
    if (p->deterministic) {
        L.oFdet = o;
        o += up(3 * (size_t)L.Npad * 8);
    } else {
        L.oF = o;
        o += up((size_t)L.Npad * 16);
    }
    L.oU = o;
    o += up((size_t)L.Npad * 16);
    L.oMarks = o;
    o += up(2 * (size_t)L.n_tiles * 4);
    L.oList = o;
    o += up(2 * (size_t)L.n_tiles * 4);
    L.oCount = o;
    o += up(4 * 4);
    L.bytes[1] = o;
    const int M = s ? s->n_nodes : 0, T = s ? s->n_tris : 0, B = s ? s->n_beads : 0, S = s ? s->n_swimmers : 0;
    o = 0;
    L.orx = o; o += up((size_t)M * 8 + 8);
    L.ory = o; o += up((size_t)M * 8 + 8);
    L.orz = o; o += up((size_t)M * 8 + 8);
    L.onf = o; o += up((size_t)M * 16 + 16);
    L.onv = o; o += up((size_t)M * 16 + 16);
    long long E = 0;  // bending edges: 3/2 per triangle of a closed bead with a bending modulus
    bool vol = false;
    for (int b = 0; b < B; ++b) {
        if (s->beads[b].kb > 0.0) E += 3ll * s->beads[b].tri_count / 2;
        vol |= s->beads[b].kv > 0.0;
    }
    L.n_edges = (int)E;
    L.otf = o; o += up(((size_t)3 * T + 4 * (size_t)E) * 16 + 16);
    L.otri = o; o += up((size_t)T * sizeof(TriDev) + 16);
    L.ocp = o; o += up((size_t)(M + 1) * 4);
    L.oce = o; o += up(((size_t)3 * T + 4 * (size_t)E) * 4 + 4);
    L.oedge = o; o += up((size_t)E * sizeof(EdgeDev) + 16);
    L.ovg = o; o += up((vol ? (size_t)3 * T : 0) * 16 + 16);
    L.ovfix = o; o += up((size_t)B * 8 + 16);
    L.onb = o; o += up((size_t)M * 4 + 4);
    L.obead = o; o += up((size_t)B * sizeof(BeadDev) + 16);
    L.oswim = o; o += up((size_t)S * sizeof(SwimDev) + 16);
    L.obd = o; o += up((size_t)B * 32 + 32);
    L.obe = o; o += up((size_t)B * 16 + 16);
    L.octl = o; o += up(sizeof(Control));
    L.osws = o; o += up((size_t)S * sizeof(lbib_swimmer_state) + 16);
    L.oxcm = o; o += up((size_t)S * 24 + 24);
    L.oswp = o; o += up((size_t)S * 64 + 64);
    L.obv = o; o += up((size_t)B * 16 + 16);
    L.obacc = o; o += up((size_t)B * 24 + 24);
    L.otrk = o; o += up((size_t)LBIB_TRACK_STEPS * S * sizeof(lbib_track_point) + 16);
    L.bytes[2] = o;
    return L;
}

}  // namespace

bool lbib::check_params(const lb_params *p, std::string &why) { return valid_params(p, why); }
bool lbib::check_structure(const lb_params *p, const lbib_structure *s, std::string &why) {
    return valid_structure(p, s, why);
}

struct lbib_ctx {
    lb_params p;
    Layout L;
    DevCtx d;
    cudaStream_t user = nullptr;   // caller stream: the fluid update of unmarked tiles and every other call
    cudaStream_t ib = nullptr;     // immersed-boundary chain of a step, concurrent with the fluid update
    cudaStream_t cap = nullptr;    // private streams used only to capture graphs
    cudaStream_t cap_ib = nullptr;
    cudaEvent_t e_fork = nullptr, e_main = nullptr, e_ib = nullptr;  // step-to-step dependencies
    cudaGraphExec_t graph = nullptr;  // GRAPH_STEPS steps from an even step
    long long step = 0;            // host mirror of the device step counter
    bool profiling = false;
    std::vector<cudaEvent_t> ev;   // event pairs around fluid-kernel launches
    size_t ev_used = 0;
    // the 16-step graph with an event-record node before and after every main
    // fluid launch (timed replays of the production schedule); its nodes in
    // capture order, re-pointed at fresh events for every replay
    cudaGraph_t tgraph_src = nullptr;
    cudaGraphExec_t tgraph = nullptr;
    std::vector<cudaGraphNode_t> tnodes;
    bool capturing_timed = false;
    Control *h_ctl = nullptr;      // pinned
    lbib_swimmer_state *h_sws = nullptr;  // pinned
    int n_nodes = 0, n_swimmers = 0;
    lbib_batch *batch = nullptr;   // set while the context belongs to a batch
    void *buf[LBIB_NBUF] = {nullptr, nullptr, nullptr};  // the caller buffers
};

struct lbib_batch {
    std::vector<lbib_ctx *> ctx;
    BatchDev bt;
    std::vector<ClassArgs> classes;  // boxes grouped by size for the main fluid launches
    void *dev = nullptr;           // device copy of the descriptors and prefix tables
    int storage = 0, forcing = 0, kernel = 0, det = 0;
    bool any_nodes = false;
    cudaStream_t user = nullptr, ib = nullptr, cap = nullptr, cap_ib = nullptr;
    cudaEvent_t e_fork = nullptr, e_main = nullptr, e_ib = nullptr;
    cudaGraphExec_t graph = nullptr;
    long long step = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    std::vector<int> class_cpt;    // cells per thread of each class's main fluid launch
    // autotuning: events around every class launch (class index, start, end)
    bool class_timing = false;
    std::vector<cudaEvent_t> tev;
    std::vector<int> tev_class;
    size_t tev_used = 0;
};

namespace {

// the update of every unmarked tile
cudaError_t main_fluid(lbib_ctx *c, bool odd, cudaStream_t s) {
    return launch_lb_main(c->d, c->p.storage, c->p.forcing, odd, s);
}

cudaError_t timed_event(lbib_ctx *c, cudaStream_t s) {
    cudaError_t e;
    while (c->ev.size() < c->ev_used + 1) {
        cudaEvent_t ev;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return e;
        c->ev.push_back(ev);
    }
    // inside the capture of the timed graph: an event-record node
    if ((e = cudaEventRecordWithFlags(c->ev[c->ev_used], s, c->capturing_timed ? cudaEventRecordExternal : 0)) !=
        cudaSuccess)
        return e;
    c->ev_used += 1;
    return cudaSuccess;
}

// Order the immersed-boundary stream after everything queued on the main stream.
cudaError_t fork(lbib_ctx *c, cudaStream_t sm, cudaStream_t sib) {
    cudaError_t e;
    if ((e = cudaEventRecord(c->e_fork, sm)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(sib, c->e_fork, 0)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(c->e_main, sm)) != cudaSuccess) return e;
    return cudaEventRecord(c->e_ib, sm);
}

// Order the main stream after the immersed-boundary stream.
cudaError_t join(lbib_ctx *c, cudaStream_t sm) { return cudaStreamWaitEvent(sm, c->e_ib, 0); }

// One coupled step on two streams (between fork and join).  Main stream: the
// fluid update of every unmarked tile (the bulk of the bytes).  IB stream,
// concurrently: forces and spreading, the fluid update of the marked tiles,
// interpolation and advection, then the marks for the next step (other
// parity).  The main stream's next step waits for this step's IB chain
// (populations of marked tiles and the next marks); the IB stream's fluid
// update waits for the previous step's main-stream update.
cudaError_t enqueue_step(lbib_ctx *c, bool odd, cudaStream_t sm, cudaStream_t sib, bool timed = false) {
    cudaError_t e;
    const int p = odd ? 1 : 0;
    if (c->n_nodes == 0) {
        if (timed && (e = timed_event(c, sm)) != cudaSuccess) return e;
        if ((e = main_fluid(c, odd, sm)) != cudaSuccess) return e;
        if (timed && (e = timed_event(c, sm)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    if ((e = cudaStreamWaitEvent(sm, c->e_ib, 0)) != cudaSuccess) return e;
    if (timed && (e = timed_event(c, sm)) != cudaSuccess) return e;
    if ((e = main_fluid(c, odd, sm)) != cudaSuccess) return e;
    if (timed && (e = timed_event(c, sm)) != cudaSuccess) return e;
    if ((e = launch_ib_prepare(c->d, sib)) != cudaSuccess) return e;
    if ((e = launch_ib_gather_spread(c->d, c->p.kernel, sib)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(sib, c->e_main, 0)) != cudaSuccess) return e;  // previous step's main update
    if ((e = cudaEventRecord(c->e_main, sm)) != cudaSuccess) return e;
    if ((e = launch_lb_marked(c->d, c->p.storage, c->p.forcing, odd, sib)) != cudaSuccess) return e;
    if ((e = launch_ib_interp(c->d, c->p.kernel, true, nullptr, 1 - p, sib)) != cudaSuccess) return e;
    return cudaEventRecord(c->e_ib, sib);
}

// Capture n coupled steps, the first of parity p0, into an executable graph
// whose nodes keep the priorities of the streams they were captured on.
cudaError_t capture_steps(lbib_ctx *c, int p0, int n, cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return ce;
    ce = fork(c, c->cap, c->cap_ib);
    for (int k = 0; k < n && ce == cudaSuccess; ++k) ce = enqueue_step(c, ((p0 + k) & 1) != 0, c->cap, c->cap_ib);
    if (ce == cudaSuccess) ce = join(c, c->cap);
    const cudaError_t ee = cudaStreamEndCapture(c->cap, &g);
    if (ce == cudaSuccess) ce = ee;
    if (ce == cudaSuccess) ce = cudaGraphInstantiateWithFlags(out, g, cudaGraphInstantiateFlagUseNodePriority);
    if (g) cudaGraphDestroy(g);
    return ce;
}

// Capture the timed 16-step graph (from an even step): the events of the
// capture are ev[0 .. 2 * GRAPH_STEPS), and tnodes[k] is the node that records ev[k].
cudaError_t capture_timed(lbib_ctx *c) {
    cudaGraph_t g = nullptr;
    c->ev_used = 0;
    c->capturing_timed = true;
    cudaError_t ce = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        ce = fork(c, c->cap, c->cap_ib);
        for (int k = 0; k < GRAPH_STEPS && ce == cudaSuccess; ++k) ce = enqueue_step(c, (k & 1) != 0, c->cap, c->cap_ib, true);
        if (ce == cudaSuccess) ce = join(c, c->cap);
        const cudaError_t ee = cudaStreamEndCapture(c->cap, &g);
        if (ce == cudaSuccess) ce = ee;
    }
    c->capturing_timed = false;
    const size_t n_ev = c->ev_used;
    c->ev_used = 0;
    if (ce == cudaSuccess && n_ev == 0) ce = cudaErrorInvalidValue;  // no fluid launch to time
    size_t n = 0;
    if (ce == cudaSuccess) ce = cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (ce == cudaSuccess && n) ce = cudaGraphGetNodes(g, nodes.data(), &n);
    c->tnodes.assign(n_ev, nullptr);
    for (size_t i = 0; i < n && ce == cudaSuccess; ++i) {
        cudaGraphNodeType t;
        if ((ce = cudaGraphNodeGetType(nodes[i], &t)) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev = nullptr;
        if ((ce = cudaGraphEventRecordNodeGetEvent(nodes[i], &ev)) != cudaSuccess) break;
        for (size_t k = 0; k < n_ev; ++k)
            if (c->ev[k] == ev) c->tnodes[k] = nodes[i];
    }
    for (size_t k = 0; k < n_ev && ce == cudaSuccess; ++k)
        if (!c->tnodes[k]) ce = cudaErrorInvalidValue;
    if (ce == cudaSuccess) ce = cudaGraphInstantiateWithFlags(&c->tgraph, g, cudaGraphInstantiateFlagUseNodePriority);
    if (ce == cudaSuccess) {
        c->tgraph_src = g;
    } else {
        if (g) cudaGraphDestroy(g);
        c->tnodes.clear();
    }
    return ce;
}

// Replay the timed graph with fresh events for this replay's launches.
cudaError_t launch_timed(lbib_ctx *c) {
    cudaError_t e;
    const size_t n = c->tnodes.size();
    while (c->ev.size() < c->ev_used + n) {
        cudaEvent_t ev;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return e;
        c->ev.push_back(ev);
    }
    for (size_t k = 0; k < n; ++k)
        if ((e = cudaGraphExecEventRecordNodeSetEvent(c->tgraph, c->tnodes[k], c->ev[c->ev_used + k])) != cudaSuccess)
            return e;
    if ((e = cudaGraphLaunch(c->tgraph, c->user)) != cudaSuccess) return e;
    c->ev_used += n;
    return cudaSuccess;
}

// Stamp the tiles of the current positions for the current step (after the
// positions are set from outside); tiles stamped before stay listed, harmlessly.
cudaError_t remark(lbib_ctx *c) {
    if (c->n_nodes == 0) return cudaSuccess;
    return launch_ib_mark(c->d, c->p.kernel, c->user);
}

int check_device_errors(lbib_ctx *c) {
    CU(cudaMemcpyAsync(c->h_ctl, c->d.ctl, sizeof(Control), cudaMemcpyDeviceToHost, c->user));
    CU(cudaStreamSynchronize(c->user));
    const int e = c->h_ctl->err;
    if (e & ERR_NONFINITE) return fail(LBIB_ENONFINITE, "non-finite density, velocity or node position");
    if (e & ERR_UNSTABLE) return fail(LBIB_EUNSTABLE, "a node moved faster than 0.1 lattice units per step");
    if (e & ERR_TIMEOUT) return fail(LBIB_ETIMEOUT, "a bounded device wait gave up");
    if (e & ERR_MARK)
        return fail(LBIB_EUNSTABLE, "a node left the region marked around its bead (membrane deformed by more than 1 lattice unit)");
    return LBIB_OK;
}

// index of direction i's value for cell (x,y,z) in the storage, given the parity of the next step
inline size_t slot_of(const lbib_ctx *c, int i, long long x, long long y, long long z, bool odd) {
    const long long nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    if (!odd) return (size_t)i * c->L.Npad + (size_t)(x + nx * (y + ny * z));
    const long long xs = (x - cx(i) + nx) % nx, ys = (y - cy(i) + ny) % ny, zs = (z - cz(i) + nz) % nz;
    return (size_t)opp(i) * c->L.Npad + (size_t)(xs + nx * (ys + ny * zs));
}

float store_scale(const lb_params *p) { return p->store_scale > 0.0 ? (float)p->store_scale : 4096.0f; }

}  // namespace

extern "C" {

const char *lbib_version(void) { return "lbib 0.1 (sm_103a)"; }

const char *lbib_strerror(int s) {
    switch (s) {
        case LBIB_OK: return "ok";
        case LBIB_EINVAL: return "invalid argument";
        case LBIB_ECUDA: return "CUDA runtime error";
        case LBIB_ENONFINITE: return "non-finite value in the simulation state";
        case LBIB_EUNSTABLE: return "node speed above 0.1 lattice units per step";
        case LBIB_ETIMEOUT: return "device-side wait timed out";
        case LBIB_ESIZE: return "buffer too small or size above a limit";
        default: return "unknown status";
    }
}

const char *lbib_last_error(void) { return g_last_error.c_str(); }

int lbib_lattice(int *c, double *w) {
    if (!c || !w) return fail(LBIB_EINVAL, "lbib_lattice: NULL output");
    for (int i = 0; i < Q; ++i) {
        c[3 * i + 0] = cx(i);
        c[3 * i + 1] = cy(i);
        c[3 * i + 2] = cz(i);
        w[i] = wgt_d(i);
    }
    return LBIB_OK;
}

int lbib_required_sizes(const lb_params *p, const lbib_structure *s, size_t *out) {
    std::string why;
    if (!out) return fail(LBIB_EINVAL, "out_bytes is NULL");
    if (!valid_params(p, why) || !valid_structure(p, s, why)) return fail(LBIB_EINVAL, why);
    Layout L = make_layout(p, s);
    for (int k = 0; k < LBIB_NBUF; ++k) out[k] = L.bytes[k];
    return LBIB_OK;
}

int lb_init(const lb_params *p, const lbib_structure *s, const lbib_buffers *b, void *stream, lbib_ctx **out) {
    std::string why;
    if (!out) return fail(LBIB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!valid_params(p, why) || !valid_structure(p, s, why)) return fail(LBIB_EINVAL, why);
    if (!b || !b->pops || !b->fields || !b->aux) return fail(LBIB_EINVAL, "a buffer pointer is NULL");
    if (((uintptr_t)b->pops | (uintptr_t)b->fields | (uintptr_t)b->aux) % ALIGN)
        return fail(LBIB_EINVAL, "buffers must be 256-byte aligned");
    const int M = s ? s->n_nodes : 0, T = s ? s->n_tris : 0, B = s ? s->n_beads : 0, S = s ? s->n_swimmers : 0;
    Layout L = make_layout(p, s);

    // mesh preprocessing on the host (reference shapes, node -> triangle lists)
    std::vector<TriDev> tri(T);
    const int E = L.n_edges;
    std::vector<int> cptr(M + 1, 0), cent(3 * (size_t)T + 4 * (size_t)E), nbead(M, 0);
    std::vector<EdgeDev> edges;
    edges.reserve(E);
    bool has_volume = false;
    std::vector<BeadDev> beads(B);
    std::vector<SwimDev> swims(S);
    for (int bi = 0; bi < B; ++bi) {
        const lbib_bead &bd = s->beads[bi];
        beads[bi].node_start = bd.node_start;
        beads[bi].node_count = bd.node_count;
        beads[bi].inv_count = (float)(1.0 / bd.node_count);
        beads[bi].pad = 0;
        beads[bi].pad2 = 0.0;
        beads[bi].kv = (float)bd.kv;
        beads[bi].V0 = 0.0;
        if (bd.kv > 0.0) {
            // enclosed volume of the rest shape (divergence theorem, outward triangles),
            // about the first node of the bead
            const double *X = s->rest_nodes, *o = X + 3 * bd.node_start;
            double V = 0.0;
            for (int t = bd.tri_start; t < bd.tri_start + bd.tri_count; ++t) {
                const int *v = s->tris + 3 * t;
                double p[3][3];
                for (int q = 0; q < 3; ++q)
                    for (int a = 0; a < 3; ++a) p[q][a] = X[3 * v[q] + a] - o[a];
                V += (p[0][0] * (p[1][1] * p[2][2] - p[1][2] * p[2][1]) + p[0][1] * (p[1][2] * p[2][0] - p[1][0] * p[2][2]) +
                      p[0][2] * (p[1][0] * p[2][1] - p[1][1] * p[2][0])) / 6.0;
            }
            if (!(V > 0.0)) return fail(LBIB_EINVAL, "a bead with a volume penalty encloses no positive volume");
            beads[bi].V0 = V;
            has_volume = true;
        }
        if (bd.kb > 0.0) {
            // bending edges with the rest angle between their triangles' normals
            const double *X = s->rest_nodes;
            for (const auto &q : bending_edges(s, bd)) {
                double P[4][3];
                for (int k = 0; k < 4; ++k)
                    for (int a = 0; a < 3; ++a) P[k][a] = X[3 * q[k] + a];
                double e[3], u[3], w[3], n1[3], n2[3];
                for (int a = 0; a < 3; ++a) {
                    e[a] = P[1][a] - P[0][a];  // b - a
                    u[a] = P[2][a] - P[0][a];  // c - a
                    w[a] = P[3][a] - P[1][a];  // d - b
                }
                // N1 = e x (c - a), N2 = (d - b) x e
                n1[0] = e[1] * u[2] - e[2] * u[1];
                n1[1] = e[2] * u[0] - e[0] * u[2];
                n1[2] = e[0] * u[1] - e[1] * u[0];
                n2[0] = w[1] * e[2] - w[2] * e[1];
                n2[1] = w[2] * e[0] - w[0] * e[2];
                n2[2] = w[0] * e[1] - w[1] * e[0];
                const double l1 = std::sqrt(n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2]);
                const double l2 = std::sqrt(n2[0] * n2[0] + n2[1] * n2[1] + n2[2] * n2[2]);
                const double le = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
                if (!(l1 > 0.0 && l2 > 0.0 && le > 0.0)) return fail(LBIB_EINVAL, "degenerate rest triangle");
                double cth = 0.0, sth = 0.0;
                for (int a = 0; a < 3; ++a) cth += n1[a] * n2[a] / (l1 * l2);
                // sin: (n1 x n2) . e / |e|
                const double cx = n1[1] * n2[2] - n1[2] * n2[1], cy = n1[2] * n2[0] - n1[0] * n2[2],
                             cz = n1[0] * n2[1] - n1[1] * n2[0];
                sth = (cx * e[0] + cy * e[1] + cz * e[2]) / (l1 * l2 * le);
                EdgeDev ed;
                for (int k = 0; k < 4; ++k) ed.v[k] = q[k];
                ed.c0 = (float)cth;
                ed.s0 = (float)sth;
                ed.kb = (float)(2.0 * std::sqrt(3.0) * bd.kb);
                ed.pad = 0;
                edges.push_back(ed);
            }
        }
        {
            // reach: largest rest distance of a node from the bead centre, plus a
            // margin of 1 lattice unit for membrane deformation
            double m[3] = {0.0, 0.0, 0.0};
            for (int j = bd.node_start; j < bd.node_start + bd.node_count; ++j)
                for (int a = 0; a < 3; ++a) m[a] += s->rest_nodes[3 * j + a];
            for (int a = 0; a < 3; ++a) m[a] /= bd.node_count;
            double r2 = 0.0;
            for (int j = bd.node_start; j < bd.node_start + bd.node_count; ++j) {
                double q = 0.0;
                for (int a = 0; a < 3; ++a) q += (s->rest_nodes[3 * j + a] - m[a]) * (s->rest_nodes[3 * j + a] - m[a]);
                r2 = std::max(r2, q);
            }
            beads[bi].reach = (float)(std::sqrt(r2) + 1.0);
        }
        for (int j = bd.node_start; j < bd.node_start + bd.node_count; ++j) nbead[j] = bi;
        for (int t = bd.tri_start; t < bd.tri_start + bd.tri_count; ++t) {
            const int *v = s->tris + 3 * t;
            const double *X = s->rest_nodes;
            double e1[3], e2[3];
            for (int a = 0; a < 3; ++a) {
                e1[a] = X[3 * v[1] + a] - X[3 * v[0] + a];
                e2[a] = X[3 * v[2] + a] - X[3 * v[0] + a];
            }
            TriDev &td = tri[t];
            td.G[0] = e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2];
            td.G[1] = e1[0] * e2[0] + e1[1] * e2[1] + e1[2] * e2[2];
            td.G[2] = e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2];
            const double det = td.G[0] * td.G[2] - td.G[1] * td.G[1];
            if (!(det > 0.0)) return fail(LBIB_EINVAL, "degenerate rest triangle");
            td.Gi[0] = (float)(td.G[2] / det);
            td.Gi[1] = (float)(-td.G[1] / det);
            td.Gi[2] = (float)(td.G[0] / det);
            td.K = (float)(0.5 * std::sqrt(det) * bd.Gs / det);
            td.inv_detG = (float)(1.0 / det);
            td.v[0] = v[0];
            td.v[1] = v[1];
            td.v[2] = v[2];
            td.skC = (float)bd.C;
            td.law = bd.law;
        }
    }
    if ((int)edges.size() != E) return fail(LBIB_EINVAL, "bending edge count does not match the closed surfaces");
    // node -> corner entries: its triangle corners, then its bending-edge slots
    for (int t = 0; t < T; ++t)
        for (int q = 0; q < 3; ++q) cptr[s->tris[3 * t + q] + 1]++;
    for (int e = 0; e < E; ++e)
        for (int q = 0; q < 4; ++q) cptr[edges[e].v[q] + 1]++;
    for (int j = 0; j < M; ++j) cptr[j + 1] += cptr[j];
    {
        std::vector<int> fill(cptr.begin(), cptr.end() - 1);
        for (int t = 0; t < T; ++t)
            for (int q = 0; q < 3; ++q) cent[fill[s->tris[3 * t + q]]++] = 3 * t + q;
        for (int e = 0; e < E; ++e)
            for (int q = 0; q < 4; ++q) cent[fill[edges[e].v[q]]++] = 3 * T + 4 * e + q;
    }
    for (int k = 0; k < S; ++k) {
        const lbib_swimmer &w = s->swimmers[k];
        SwimDev &d = swims[k];
        for (int q = 0; q < 3; ++q) {
            d.bead[q] = w.bead[q];
            d.amp[q] = (float)w.amp[q];
            d.phase_turns[q] = w.phase[q] / (2.0 * 3.14159265358979323846);
            beads[w.bead[q]].swimmer = k;
            beads[w.bead[q]].slot = q;
        }
        d.balance = w.balance;
        d.k = w.k_spring;
        d.L = w.L_spring;
        d.L2 = w.L_spring * w.L_spring;
        d.inv_period = 1.0 / w.period;
        d.period = w.period;
        d.pad = 0;
    }

    lbib_ctx *c = new lbib_ctx();
    c->p = *p;
    c->L = L;
    c->user = (cudaStream_t)stream;
    c->n_nodes = M;
    c->n_swimmers = S;
    DevCtx &d = c->d;
    memset(&d, 0, sizeof(d));
    d.nx = p->nx;
    d.ny = p->ny;
    d.nz = p->nz;
    d.N = L.N;
    d.Npad = L.Npad;
    d.n_tiles = L.n_tiles;
    d.tile_x = L.tile_x;
    d.tiles_x = L.tiles_x;
    // adjacent cells per fluid thread: four for 16-bit storage, two for FP32,
    // when the rows split into tiles of that many cells
    {
        int cpt = p->storage == LBIB_F32 ? 2 : 4;
        while (cpt > 1 && (L.tile_x % cpt || p->nx % cpt)) cpt /= 2;
        d.cells_per_thread = cpt < 1 ? 1 : (cpt == 3 ? 2 : cpt);
    }

    d.tau = (float)p->tau;
    d.omega = (float)(1.0 / p->tau);
    d.rho0 = (float)p->rho0;
    for (int a = 0; a < 3; ++a) d.g[a] = (float)p->g[a];
    d.has_g = (p->g[0] != 0.0 || p->g[1] != 0.0 || p->g[2] != 0.0);
    d.st_scale = store_scale(p);
    d.st_inv_scale = 1.0f / d.st_scale;
    d.n_nodes = M;
    d.n_tris = T;
    d.n_beads = B;
    d.n_swimmers = S;
    d.deterministic = p->deterministic ? 1 : 0;
    char *F = (char *)b->fields, *A = (char *)b->aux;
    c->buf[0] = b->pops;
    c->buf[1] = b->fields;
    c->buf[2] = b->aux;
    d.pops = b->pops;
    d.F = p->deterministic ? nullptr : (float4 *)(F + L.oF);
    d.Fdet = p->deterministic ? (unsigned long long *)(F + L.oFdet) : nullptr;
    d.U = (float4 *)(F + L.oU);
    d.marks = (int *)(F + L.oMarks);
    d.tile_list = (int *)(F + L.oList);
    d.tile_count = (int *)(F + L.oCount);
    d.rx = (double *)(A + L.orx);
    d.ry = (double *)(A + L.ory);
    d.rz = (double *)(A + L.orz);
    d.node_force = (float4 *)(A + L.onf);
    d.node_vel = (float4 *)(A + L.onv);
    d.tri_force = (float4 *)(A + L.otf);
    d.tris = (const TriDev *)(A + L.otri);
    d.csr_ptr = (const int *)(A + L.ocp);
    d.csr_ent = (const int *)(A + L.oce);
    d.n_edges = E;
    d.edges = (const EdgeDev *)(A + L.oedge);
    d.has_volume = has_volume ? 1 : 0;
    d.tri_vgrad = has_volume ? (float4 *)(A + L.ovg) : nullptr;
    d.bead_Vfix = (long long *)(A + L.ovfix);
    d.node_bead = (const int *)(A + L.onb);
    d.beads = (const BeadDev *)(A + L.obead);
    d.swims = (const SwimDev *)(A + L.oswim);
    d.bead_R = (double *)(A + L.obd);
    d.bead_ext = (float4 *)(A + L.obe);
    d.ctl = (Control *)(A + L.octl);
    d.sw_state = (lbib_swimmer_state *)(A + L.osws);
    d.xcm0 = (double *)(A + L.oxcm);
    d.sw_period = (double *)(A + L.oswp);
    d.bead_V = (float4 *)(A + L.obv);
    d.bead_acc = (unsigned long long *)(A + L.obacc);
    d.track = (lbib_track_point *)(A + L.otrk);

    auto bail = [&](int code) {
        lb_destroy(c);
        return code;
    };
    if (cudaMallocHost(&c->h_ctl, sizeof(Control)) != cudaSuccess ||
        cudaMallocHost(&c->h_sws, sizeof(lbib_swimmer_state) * (S > 0 ? S : 1)) != cudaSuccess)
        return bail(fail(LBIB_ECUDA, "cudaMallocHost failed"));
    cudaStream_t u = c->user;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return bail(fail(LBIB_ECUDA, "querying the device failed"));
        // persistent grid of the marked-tile fluid kernel: one block per SM
        d.marked_grid = sms;
    }
    // rest state: all deviations zero, fields, marks and lists zero
    if (cudaMemsetAsync(b->pops, 0, L.bytes[0], u) != cudaSuccess || cudaMemsetAsync(b->fields, 0, L.bytes[1], u) != cudaSuccess ||
        cudaMemsetAsync(b->aux, 0, L.bytes[2], u) != cudaSuccess ||
        // stamps -1 (never marked); generations a different negative value, so no
        // tile counts as marked until a step stamps it
        cudaMemsetAsync(d.marks, 0xff, 2 * (size_t)L.n_tiles * 4, u) != cudaSuccess ||
        cudaMemsetAsync((char *)d.ctl + offsetof(Control, gen), 0xfe, sizeof(int) * 2, u) != cudaSuccess)
        return bail(fail(LBIB_ECUDA, "cudaMemsetAsync failed"));
    std::vector<double> sx(M), sy(M), sz(M);
    for (int j = 0; j < M; ++j) {
        sx[j] = s->rest_nodes[3 * j];
        sy[j] = s->rest_nodes[3 * j + 1];
        sz[j] = s->rest_nodes[3 * j + 2];
    }
    auto h2d = [&](void *dst, const void *src, size_t n) {
        return n == 0 || cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, u) == cudaSuccess;
    };
    bool ok = h2d(d.rx, sx.data(), M * 8) && h2d(d.ry, sy.data(), M * 8) && h2d(d.rz, sz.data(), M * 8) &&
              h2d((void *)d.tris, tri.data(), T * sizeof(TriDev)) && h2d((void *)d.csr_ptr, cptr.data(), (M + 1) * 4) &&
              h2d((void *)d.csr_ent, cent.data(), cent.size() * 4) && h2d((void *)d.node_bead, nbead.data(), M * 4) &&
              h2d((void *)d.edges, edges.data(), edges.size() * sizeof(EdgeDev)) &&
              h2d((void *)d.beads, beads.data(), B * sizeof(BeadDev)) && h2d((void *)d.swims, swims.data(), S * sizeof(SwimDev));
    if (!ok) return bail(fail(LBIB_ECUDA, "uploading mesh tables failed"));
    if (launch_bead_init(d, u) != cudaSuccess || launch_swimmer_state(d, true, u) != cudaSuccess ||
        launch_ib_mark(d, p->kernel, u) != cudaSuccess)
        return bail(fail(LBIB_ECUDA, "bead initialisation launch failed"));
    if (cudaStreamSynchronize(u) != cudaSuccess) return bail(fail(LBIB_ECUDA, "init synchronisation failed"));
    if (M > 0) {
        // size the marked-tile kernel's grid to the tiles the stencils mark now,
        // with room for the swimmers to move into new tiles (more are handled in a loop)
        int cnt = 0;
        if (cudaMemcpy(&cnt, d.tile_count, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            return bail(fail(LBIB_ECUDA, "reading the marked-tile count failed"));
        d.marked_grid = std::min(L.n_tiles, std::max(32, cnt + cnt / 4 + 16));
    }

    // streams and events of the two-stream step; the IB stream gets the
    // highest priority so its small kernels are scheduled between fluid blocks
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->ib, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->cap_ib, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->e_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->e_main, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->e_ib, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(LBIB_ECUDA, "creating streams or events failed"));

    // capture GRAPH_STEPS coupled steps (alternating AA parity) into one graph
    cudaError_t ce = capture_steps(c, 0, GRAPH_STEPS, &c->graph);
    if (ce != cudaSuccess) return bail(fail(LBIB_ECUDA, std::string("graph capture failed: ") + cudaGetErrorString(ce)));
    *out = c;
    return LBIB_OK;
}

int lb_step(lbib_ctx *c, long long n) {
    if (!c) return fail(LBIB_EINVAL, "ctx is NULL");
    if (c->batch) return fail(LBIB_EINVAL, "the context belongs to a batch: advance it with lb_batch_step");
    if (n < 0) return fail(LBIB_EINVAL, "n_steps < 0");
    bool forked = false;
    const bool graphs = use_graphs(c->L.N);
    while (n > 0) {
        if (graphs && c->profiling && c->tgraph && (c->step & 1) == 0 && n >= GRAPH_STEPS) {
            if (forked) {
                CU(join(c, c->user));
                forked = false;
            }
            CU(launch_timed(c));
            c->step += GRAPH_STEPS;
            n -= GRAPH_STEPS;
        } else if (graphs && !c->profiling && (c->step & 1) == 0 && n >= GRAPH_STEPS) {
            if (forked) {
                CU(join(c, c->user));
                forked = false;
            }
            CU(cudaGraphLaunch(c->graph, c->user));
            c->step += GRAPH_STEPS;
            n -= GRAPH_STEPS;
        } else {
            if (!forked) {
                CU(fork(c, c->user, c->ib));
                forked = true;
            }
            CU(enqueue_step(c, (c->step & 1) != 0, c->user, c->ib, c->profiling));
            c->step += 1;
            n -= 1;
        }
    }
    if (forked) CU(join(c, c->user));
    return LBIB_OK;
}

int ib_spread(lbib_ctx *c) {
    if (!c) return fail(LBIB_EINVAL, "ctx is NULL");
    if (c->n_nodes == 0) return LBIB_OK;
    CU(launch_ib_prepare(c->d, c->user));
    CU(launch_ib_gather_spread(c->d, c->p.kernel, c->user));
    return LBIB_OK;
}

int ib_interpolate(lbib_ctx *c, float *vel) {
    if (!c) return fail(LBIB_EINVAL, "ctx is NULL");
    if (c->n_nodes == 0) return LBIB_OK;
    if (!vel) return fail(LBIB_EINVAL, "node_vel_out is NULL");
    CU(launch_ib_interp(c->d, c->p.kernel, false, vel, -1, c->user));
    return LBIB_OK;
}

int swimmer_state(lbib_ctx *c, int s, lbib_swimmer_state *out) {
    if (!c || !out) return fail(LBIB_EINVAL, "NULL argument");
    if (s < 0 || s >= c->n_swimmers) return fail(LBIB_EINVAL, "swimmer index out of range");
    CU(launch_swimmer_state(c->d, false, c->user));
    CU(cudaMemcpyAsync(c->h_sws + s, c->d.sw_state + s, sizeof(lbib_swimmer_state), cudaMemcpyDeviceToHost, c->user));
    int st = check_device_errors(c);
    *out = c->h_sws[s];
    return st;
}

int swimmer_state_async(lbib_ctx *c, lbib_swimmer_state *out) {
    if (!c || (!out && c->n_swimmers)) return fail(LBIB_EINVAL, "NULL argument");
    if (c->n_swimmers == 0) return LBIB_OK;
    CU(launch_swimmer_state(c->d, false, c->user));
    CU(cudaMemcpyAsync(out, c->d.sw_state, sizeof(lbib_swimmer_state) * c->n_swimmers, cudaMemcpyDeviceToHost, c->user));
    return LBIB_OK;
}

int lb_track(lbib_ctx *c, long long n, lbib_track_point *out) {
    if (!c || (!out && c->n_swimmers)) return fail(LBIB_EINVAL, "NULL argument");
    if (n < 1 || n > LBIB_TRACK_STEPS) return fail(LBIB_EINVAL, "n_steps outside [1, LBIB_TRACK_STEPS]");
    if (n > c->step) return fail(LBIB_EINVAL, "n_steps exceeds the steps taken since lb_init");
    if (c->n_swimmers == 0) return LBIB_OK;
    cudaStream_t s = c->batch ? c->batch->user : c->user;
    const size_t S = (size_t)c->n_swimmers;
    // step t (1-based) lives in slot (t - 1) mod LBIB_TRACK_STEPS: at most two contiguous runs
    const long long first = (c->step - n) % LBIB_TRACK_STEPS;
    const long long run = std::min<long long>(n, LBIB_TRACK_STEPS - first);
    CU(cudaMemcpyAsync(out, c->d.track + first * S, run * S * sizeof(lbib_track_point), cudaMemcpyDeviceToHost, s));
    if (run < n)
        CU(cudaMemcpyAsync(out + run * S, c->d.track, (n - run) * S * sizeof(lbib_track_point), cudaMemcpyDeviceToHost, s));
    return LBIB_OK;
}

int lb_sync(lbib_ctx *c) {
    if (!c) return fail(LBIB_EINVAL, "ctx is NULL");
    return check_device_errors(c);
}

int lb_get_macros(lbib_ctx *c, float *rho, float *u) {
    if (!c || !rho || !u) return fail(LBIB_EINVAL, "NULL argument");
    CU(launch_lb_macros(c->d, c->p.storage, (c->step & 1) != 0, rho, u, c->user));
    return LBIB_OK;
}

int lb_get_populations(lbib_ctx *c, double *hf) {
    if (!c || !hf) return fail(LBIB_EINVAL, "NULL argument");
    const size_t n = c->L.bytes[0];
    std::vector<unsigned char> raw(n);
    CU(cudaMemcpyAsync(raw.data(), c->d.pops, n, cudaMemcpyDeviceToHost, c->user));
    CU(cudaStreamSynchronize(c->user));
    const bool odd = (c->step & 1) != 0;
    const long long nx = c->p.nx, ny = c->p.ny, nz = c->p.nz, N = c->L.N;
    const float sc = store_scale(&c->p);
    for (int i = 0; i < Q; ++i)
        for (long long z = 0; z < nz; ++z)
            for (long long y = 0; y < ny; ++y)
                for (long long x = 0; x < nx; ++x) {
                    const size_t k = slot_of(c, i, x, y, z, odd);
                    double dv;
                    if (c->p.storage == LBIB_F32) dv = ((const float *)raw.data())[k];
                    else if (c->p.storage == LBIB_F16) dv = (double)__half2float(((const __half *)raw.data())[k]) * wgt_d(i) / sc;
                    else dv = (double)__bfloat162float(((const __nv_bfloat16 *)raw.data())[k]) * wgt_d(i) / sc;
                    hf[(size_t)i * N + x + nx * (y + ny * z)] = wgt_d(i) * c->p.rho0 + dv;
                }
    return LBIB_OK;
}

int lb_set_populations(lbib_ctx *c, const double *hf) {
    if (!c || !hf) return fail(LBIB_EINVAL, "NULL argument");
    const size_t n = c->L.bytes[0];
    std::vector<unsigned char> raw(n, 0);
    const bool odd = (c->step & 1) != 0;
    const long long nx = c->p.nx, ny = c->p.ny, nz = c->p.nz, N = c->L.N;
    const float sc = store_scale(&c->p);
    for (int i = 0; i < Q; ++i)
        for (long long z = 0; z < nz; ++z)
            for (long long y = 0; y < ny; ++y)
                for (long long x = 0; x < nx; ++x) {
                    const size_t k = slot_of(c, i, x, y, z, odd);
                    const double dv = hf[(size_t)i * N + x + nx * (y + ny * z)] - wgt_d(i) * c->p.rho0;
                    if (c->p.storage == LBIB_F32) ((float *)raw.data())[k] = (float)dv;
                    else if (c->p.storage == LBIB_F16) ((__half *)raw.data())[k] = __float2half_rn((float)(dv / wgt_d(i) * sc));
                    else ((__nv_bfloat16 *)raw.data())[k] = __float2bfloat16_rn((float)(dv / wgt_d(i) * sc));
                }
    CU(cudaMemcpyAsync(c->d.pops, raw.data(), n, cudaMemcpyHostToDevice, c->user));
    CU(cudaStreamSynchronize(c->user));
    return LBIB_OK;
}

int lb_get_nodes(lbib_ctx *c, double *h) {
    if (!c || (!h && c->n_nodes)) return fail(LBIB_EINVAL, "NULL argument");
    const int M = c->n_nodes;
    if (M == 0) return LBIB_OK;
    std::vector<double> x(M), y(M), z(M);
    CU(cudaMemcpyAsync(x.data(), c->d.rx, M * 8, cudaMemcpyDeviceToHost, c->user));
    CU(cudaMemcpyAsync(y.data(), c->d.ry, M * 8, cudaMemcpyDeviceToHost, c->user));
    CU(cudaMemcpyAsync(z.data(), c->d.rz, M * 8, cudaMemcpyDeviceToHost, c->user));
    CU(cudaStreamSynchronize(c->user));
    for (int j = 0; j < M; ++j) {
        h[3 * j] = x[j];
        h[3 * j + 1] = y[j];
        h[3 * j + 2] = z[j];
    }
    return LBIB_OK;
}

int lb_set_nodes(lbib_ctx *c, const double *h) {
    if (!c || (!h && c->n_nodes)) return fail(LBIB_EINVAL, "NULL argument");
    const int M = c->n_nodes;
    if (M == 0) return LBIB_OK;
    std::vector<double> x(M), y(M), z(M);
    for (int j = 0; j < M; ++j) {
        if (!std::isfinite(h[3 * j]) || !std::isfinite(h[3 * j + 1]) || !std::isfinite(h[3 * j + 2]))
            return fail(LBIB_EINVAL, "non-finite node coordinate");
        x[j] = h[3 * j];
        y[j] = h[3 * j + 1];
        z[j] = h[3 * j + 2];
    }
    CU(cudaMemcpyAsync(c->d.rx, x.data(), M * 8, cudaMemcpyHostToDevice, c->user));
    CU(cudaMemcpyAsync(c->d.ry, y.data(), M * 8, cudaMemcpyHostToDevice, c->user));
    CU(cudaMemcpyAsync(c->d.rz, z.data(), M * 8, cudaMemcpyHostToDevice, c->user));
    CU(launch_bead_init(c->d, c->user));
    CU(remark(c));
    CU(cudaStreamSynchronize(c->user));
    return LBIB_OK;
}

int ib_get_node_forces(lbib_ctx *c, float *h) {
    if (!c || (!h && c->n_nodes)) return fail(LBIB_EINVAL, "NULL argument");
    const int M = c->n_nodes;
    if (M == 0) return LBIB_OK;
    std::vector<float4> v(M);
    CU(cudaMemcpyAsync(v.data(), c->d.node_force, M * 16, cudaMemcpyDeviceToHost, c->user));
    CU(cudaStreamSynchronize(c->user));
    for (int j = 0; j < M; ++j) {
        h[3 * j] = v[j].x;
        h[3 * j + 1] = v[j].y;
        h[3 * j + 2] = v[j].z;
    }
    return LBIB_OK;
}

int lb_get_force_field(lbib_ctx *c, float *h) {
    if (!c || !h) return fail(LBIB_EINVAL, "NULL argument");
    const long long N = c->L.N, Np = c->L.Npad;
    if (c->p.deterministic) {
        std::vector<long long> v(3 * (size_t)Np);
        CU(cudaMemcpyAsync(v.data(), c->d.Fdet, 3 * (size_t)Np * 8, cudaMemcpyDeviceToHost, c->user));
        CU(cudaStreamSynchronize(c->user));
        for (long long k = 0; k < N; ++k)
            for (int a = 0; a < 3; ++a) h[3 * k + a] = (float)((double)v[a * Np + k] * FIX_INV);
    } else {
        std::vector<float4> v(N);
        CU(cudaMemcpyAsync(v.data(), c->d.F, (size_t)N * 16, cudaMemcpyDeviceToHost, c->user));
        CU(cudaStreamSynchronize(c->user));
        for (long long k = 0; k < N; ++k) {
            h[3 * k] = v[k].x;
            h[3 * k + 1] = v[k].y;
            h[3 * k + 2] = v[k].z;
        }
    }
    return LBIB_OK;
}

int lb_set_velocity(lbib_ctx *c, const float *h) {
    if (!c || !h) return fail(LBIB_EINVAL, "NULL argument");
    const long long N = c->L.N;
    std::vector<float4> v(N);
    for (long long k = 0; k < N; ++k) v[k] = make_float4(h[3 * k], h[3 * k + 1], h[3 * k + 2], 0.f);
    CU(cudaMemcpyAsync(c->d.U, v.data(), (size_t)N * 16, cudaMemcpyHostToDevice, c->user));
    CU(cudaStreamSynchronize(c->user));
    return LBIB_OK;
}

int lb_profile(lbib_ctx *c, int on) {
    if (!c) return fail(LBIB_EINVAL, "ctx is NULL");
    CU(cudaStreamSynchronize(c->user));
    // timed replays of the production graph when graphs are in use
    if (on && !c->tgraph && !c->batch && use_graphs(c->L.N)) CU(capture_timed(c));
    c->profiling = on != 0;
    c->ev_used = 0;
    return LBIB_OK;
}

int lb_profile_read(lbib_ctx *c, double *total_ms, long long *launches) {
    if (!c || !total_ms || !launches) return fail(LBIB_EINVAL, "NULL argument");
    CU(cudaStreamSynchronize(c->user));
    double t = 0.0;
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]));
        t += ms;
    }
    *total_ms = t;
    *launches = (long long)(c->ev_used / 2);
    return LBIB_OK;
}

int lb_marked_cells(lbib_ctx *c, long long *cells) {
    if (!c || !cells) return fail(LBIB_EINVAL, "NULL argument");
    int cnt[2] = {0, 0};
    CU(cudaMemcpyAsync(cnt, c->d.tile_count, sizeof(cnt), cudaMemcpyDeviceToHost, c->user));
    CU(cudaStreamSynchronize(c->user));
    const long long n = (long long)cnt[c->step & 1] * c->L.tile_x;
    *cells = n < c->L.N ? n : c->L.N;
    return LBIB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- checkpoints
// Blob: header, then the three caller buffers as they are on the device (the
// populations in their stored format and AA parity; force, velocity and tile
// stamps; node positions, bead centres, mesh tables, control block and
// swimmer accumulators).  The buffers hold no pointers, so restoring them into
// a context over the same box and structure continues the run exactly.
namespace {

struct CkpHeader {
    char magic[8];  // "LBIBCKP1"
    int version;
    int nx, ny, nz, storage, forcing, kernel, deterministic;
    int n_nodes, n_tris, n_beads, n_swimmers;
    unsigned long long bytes[LBIB_NBUF];
    long long step;
    unsigned long long checksum;  // over the buffer bytes
};

// 64-bit FNV-1a over 8-byte words (then the tail bytes)
unsigned long long checksum64(const unsigned char *p, size_t n, unsigned long long h) {
    const unsigned long long prime = 1099511628211ull;
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
        unsigned long long w;
        memcpy(&w, p + i, 8);
        h = (h ^ w) * prime;
    }
    for (; i < n; ++i) h = (h ^ p[i]) * prime;
    return h;
}

void fill_header(const lbib_ctx *c, CkpHeader &h) {
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, "LBIBCKP1", 8);
    h.version = 1;
    h.nx = c->p.nx;
    h.ny = c->p.ny;
    h.nz = c->p.nz;
    h.storage = c->p.storage;
    h.forcing = c->p.forcing;
    h.kernel = c->p.kernel;
    h.deterministic = c->p.deterministic;
    h.n_nodes = c->d.n_nodes;
    h.n_tris = c->d.n_tris;
    h.n_beads = c->d.n_beads;
    h.n_swimmers = c->d.n_swimmers;
    for (int k = 0; k < LBIB_NBUF; ++k) h.bytes[k] = c->L.bytes[k];
    h.step = c->step;
}

size_t ckp_bytes(const lbib_ctx *c) {
    size_t n = sizeof(CkpHeader);
    for (int k = 0; k < LBIB_NBUF; ++k) n += c->L.bytes[k];
    return n;
}

}  // namespace

extern "C" {

int lb_checkpoint_size(lbib_ctx *c, size_t *bytes) {
    if (!c || !bytes) return fail(LBIB_EINVAL, "NULL argument");
    *bytes = ckp_bytes(c);
    return LBIB_OK;
}

int lb_checkpoint(lbib_ctx *c, void *host, size_t bytes) {
    if (!c || !host) return fail(LBIB_EINVAL, "NULL argument");
    if (bytes < ckp_bytes(c)) return fail(LBIB_ESIZE, "checkpoint buffer smaller than lb_checkpoint_size");
    const int st = check_device_errors(c);  // synchronises; a failed run is not saved
    if (st != LBIB_OK) return st;
    CkpHeader h;
    fill_header(c, h);
    unsigned char *dst = (unsigned char *)host + sizeof(CkpHeader);
    unsigned long long sum = 1469598103934665603ull;
    for (int k = 0; k < LBIB_NBUF; ++k) {
        CU(cudaMemcpy(dst, c->buf[k], c->L.bytes[k], cudaMemcpyDeviceToHost));
        sum = checksum64(dst, c->L.bytes[k], sum);
        dst += c->L.bytes[k];
    }
    h.checksum = sum;
    memcpy(host, &h, sizeof(h));
    return LBIB_OK;
}

int lb_restore(lbib_ctx *c, const void *host, size_t bytes) {
    if (!c || !host) return fail(LBIB_EINVAL, "NULL argument");
    if (c->batch) return fail(LBIB_EINVAL, "the context belongs to a batch");
    if (bytes < sizeof(CkpHeader)) return fail(LBIB_EINVAL, "not a checkpoint (too short)");
    CkpHeader h, mine;
    memcpy(&h, host, sizeof(h));
    fill_header(c, mine);
    if (memcmp(h.magic, "LBIBCKP1", 8) != 0 || h.version != 1) return fail(LBIB_EINVAL, "not a checkpoint of this format");
    mine.step = h.step;
    mine.checksum = h.checksum;
    if (memcmp(&h, &mine, sizeof(h)) != 0)
        return fail(LBIB_EINVAL, "checkpoint of a different box, storage, scheme or structure");
    if (bytes < ckp_bytes(c)) return fail(LBIB_ESIZE, "checkpoint truncated");
    const unsigned char *src = (const unsigned char *)host + sizeof(CkpHeader);
    unsigned long long sum = 1469598103934665603ull;
    size_t off = 0;
    for (int k = 0; k < LBIB_NBUF; ++k) {
        sum = checksum64(src + off, c->L.bytes[k], sum);
        off += c->L.bytes[k];
    }
    if (sum != h.checksum) return fail(LBIB_EINVAL, "checkpoint checksum mismatch (corrupted)");
    CU(cudaStreamSynchronize(c->user));
    if (c->ib) CU(cudaStreamSynchronize(c->ib));
    off = 0;
    for (int k = 0; k < LBIB_NBUF; ++k) {
        CU(cudaMemcpy(c->buf[k], src + off, c->L.bytes[k], cudaMemcpyHostToDevice));
        off += c->L.bytes[k];
    }
    c->step = h.step;
    return LBIB_OK;
}

}  // extern "C"

extern "C" {

int lb_destroy(lbib_ctx *c) {
    if (!c) return LBIB_OK;
    if (c->batch) return fail(LBIB_EINVAL, "the context belongs to a batch: destroy the batch first");
    cudaStreamSynchronize(c->user);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->ib) cudaStreamSynchronize(c->ib);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->tgraph) cudaGraphExecDestroy(c->tgraph);
    if (c->tgraph_src) cudaGraphDestroy(c->tgraph_src);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->cap_ib) cudaStreamDestroy(c->cap_ib);
    if (c->ib) cudaStreamDestroy(c->ib);
    if (c->e_fork) cudaEventDestroy(c->e_fork);
    if (c->e_main) cudaEventDestroy(c->e_main);
    if (c->e_ib) cudaEventDestroy(c->e_ib);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    if (c->h_sws) cudaFreeHost(c->h_sws);
    delete c;
    return LBIB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batches
namespace {

cudaError_t batch_timed_event(lbib_batch *b, cudaStream_t s) {
    cudaError_t e;
    while (b->ev.size() < b->ev_used + 1) {
        cudaEvent_t ev;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return e;
        b->ev.push_back(ev);
    }
    if ((e = cudaEventRecord(b->ev[b->ev_used], s)) != cudaSuccess) return e;
    b->ev_used += 1;
    return cudaSuccess;
}

cudaError_t class_event(lbib_batch *b, int cls, cudaStream_t s) {
    cudaError_t e;
    while (b->tev.size() < b->tev_used + 1) {
        cudaEvent_t ev;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return e;
        b->tev.push_back(ev);
        b->tev_class.push_back(-1);
    }
    if ((e = cudaEventRecord(b->tev[b->tev_used], s)) != cudaSuccess) return e;
    b->tev_class[b->tev_used] = cls;
    b->tev_used += 1;
    return cudaSuccess;
}

cudaError_t batch_fork(lbib_batch *b, cudaStream_t sm, cudaStream_t sib) {
    cudaError_t e;
    if ((e = cudaEventRecord(b->e_fork, sm)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(sib, b->e_fork, 0)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(b->e_main, sm)) != cudaSuccess) return e;
    return cudaEventRecord(b->e_ib, sm);
}

// The two-stream coupled step of enqueue_step, with every launch covering all boxes.
cudaError_t batch_enqueue_step(lbib_batch *b, bool odd, cudaStream_t sm, cudaStream_t sib, bool timed) {
    cudaError_t e;
    const BatchDev &bt = b->bt;
    auto main_fluid = [&]() -> cudaError_t {
        cudaError_t r;
        if (timed && (r = batch_timed_event(b, sm)) != cudaSuccess) return r;
        for (size_t k = 0; k < b->classes.size(); ++k) {
            if (b->class_timing && (r = class_event(b, (int)k, sm)) != cudaSuccess) return r;
            if ((r = launch_lb_class(b->classes[k], b->storage, b->forcing, b->class_cpt[k], odd, sm)) != cudaSuccess)
                return r;
            if (b->class_timing && (r = class_event(b, (int)k, sm)) != cudaSuccess) return r;
        }
        if (timed && (r = batch_timed_event(b, sm)) != cudaSuccess) return r;
        return cudaSuccess;
    };
    if (!b->any_nodes) return main_fluid();
    if ((e = cudaStreamWaitEvent(sm, b->e_ib, 0)) != cudaSuccess) return e;
    if ((e = main_fluid()) != cudaSuccess) return e;
    if ((e = launch_ib_batch(bt, b->kernel, b->det, 0, sib)) != cudaSuccess) return e;
    if ((e = launch_ib_batch(bt, b->kernel, b->det, 1, sib)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(sib, b->e_main, 0)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(b->e_main, sm)) != cudaSuccess) return e;
    if ((e = launch_lb_batch(bt, b->storage, b->forcing, b->det, true, odd, sib)) != cudaSuccess) return e;
    if ((e = launch_ib_batch(bt, b->kernel, b->det, 2, sib)) != cudaSuccess) return e;
    return cudaEventRecord(b->e_ib, sib);
}

// capture GRAPH_STEPS batch steps, starting at the parity of the current step
cudaError_t capture_batch_graph(lbib_batch *b) {
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    b->step = b->ctx[0]->step;
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return ce;
    ce = batch_fork(b, b->cap, b->cap_ib);
    for (int k = 0; k < GRAPH_STEPS && ce == cudaSuccess; ++k)
        ce = batch_enqueue_step(b, ((b->step + k) & 1) != 0, b->cap, b->cap_ib, false);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->cap, b->e_ib, 0);
    const cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
    if (ce == cudaSuccess) ce = ee;
    if (ce == cudaSuccess) ce = cudaGraphInstantiateWithFlags(&b->graph, g, cudaGraphInstantiateFlagUseNodePriority);
    if (g) cudaGraphDestroy(g);
    return ce;
}

// a cells-per-thread count the main fluid kernel of class k can use
bool cpt_valid(const lbib_batch *b, size_t k, int cpt) {
    const DevCtx &c = b->classes[k].box[0];
    if (b->storage == LBIB_F32 && cpt > 2) return false;
    return c.tile_x % cpt == 0 && c.nx % cpt == 0;
}

}  // namespace

extern "C" {

int lb_batch_create(lbib_ctx *const *ctxs, int n, lbib_batch **out) {
    if (!out) return fail(LBIB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1 || n > LBIB_MAX_BATCH) return fail(LBIB_EINVAL, "need 1..1024 contexts");
    const lbib_ctx *c0 = ctxs[0];
    if (!c0) return fail(LBIB_EINVAL, "a context is NULL");
    int cpt = 4;
    for (int i = 0; i < n; ++i) {
        const lbib_ctx *c = ctxs[i];
        if (!c) return fail(LBIB_EINVAL, "a context is NULL");
        if (c->batch) return fail(LBIB_EINVAL, "a context already belongs to a batch");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == c) return fail(LBIB_EINVAL, "a context appears twice");
        if (c->p.storage != c0->p.storage || c->p.forcing != c0->p.forcing || c->p.kernel != c0->p.kernel ||
            c->p.deterministic != c0->p.deterministic)
            return fail(LBIB_EINVAL, "batched contexts must share storage, forcing, kernel and determinism");
        if (c->step != c0->step) return fail(LBIB_EINVAL, "batched contexts must have taken the same number of steps");
        if (c->user != c0->user) return fail(LBIB_EINVAL, "batched contexts must use the same stream");
        cpt = std::min(cpt, c->d.cells_per_thread);
    }
    lbib_batch *b = new lbib_batch();
    auto bail = [&](int code) {
        lb_batch_destroy(b);
        return code;
    };
    b->ctx.assign(ctxs, ctxs + n);
    b->storage = c0->p.storage;
    b->forcing = c0->p.forcing;
    b->kernel = c0->p.kernel;
    b->det = c0->p.deterministic;
    b->user = c0->user;
    b->step = c0->step;
    std::vector<DevCtx> boxes(n);
    std::vector<int> om(n + 1, 0), op(n + 1, 0), og(n + 1, 0), oi(n + 1, 0);
    int max_threads = 1, marked = 0;
    for (int i = 0; i < n; ++i) {
        boxes[i] = ctxs[i]->d;
        boxes[i].cells_per_thread = cpt;
        om[i + 1] = om[i] + boxes[i].n_tiles;
        op[i + 1] = op[i] + (boxes[i].n_nodes ? ib_blocks_prepare(boxes[i]) : 0);
        og[i + 1] = og[i] + (boxes[i].n_nodes ? ib_blocks_spread(boxes[i]) : 0);
        oi[i + 1] = oi[i] + (boxes[i].n_nodes ? ib_blocks_interp(boxes[i], b->kernel) : 0);
        max_threads = std::max(max_threads, boxes[i].tile_x / cpt);
        if (boxes[i].n_nodes) {
            b->any_nodes = true;
            marked += boxes[i].marked_grid;
        }
    }
    const size_t bytes = sizeof(DevCtx) * n + 4 * sizeof(int) * (n + 1);
    if (cudaMalloc(&b->dev, bytes) != cudaSuccess) return bail(fail(LBIB_ECUDA, "cudaMalloc of the batch tables failed"));
    char *dp = (char *)b->dev;
    if (cudaMemcpy(dp, boxes.data(), sizeof(DevCtx) * n, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(fail(LBIB_ECUDA, "uploading the batch tables failed"));
    int *offs[4];
    const std::vector<int> *src[4] = {&om, &op, &og, &oi};
    for (int k = 0; k < 4; ++k) {
        offs[k] = (int *)(dp + sizeof(DevCtx) * n + k * sizeof(int) * (n + 1));
        if (cudaMemcpy(offs[k], src[k]->data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(LBIB_ECUDA, "uploading the batch tables failed"));
    }
    // size classes for the main fluid launches (at most LBIB_CLASS_BOXES boxes per launch)
    for (int i = 0; i < n; ++i) {
        ClassArgs *hit = nullptr;
        for (ClassArgs &ca : b->classes)
            if (ca.n < LBIB_CLASS_BOXES && ca.box[0].nx == boxes[i].nx && ca.box[0].ny == boxes[i].ny &&
                ca.box[0].nz == boxes[i].nz)
                hit = &ca;
        if (!hit) {
            b->classes.emplace_back();
            hit = &b->classes.back();
            memset(hit, 0, sizeof(ClassArgs));
        }
        hit->box[hit->n++] = boxes[i];
    }
    BatchDev &bt = b->bt;
    bt.n_boxes = n;
    bt.boxes = (const DevCtx *)dp;
    bt.off_main = offs[0];
    bt.off_prep = offs[1];
    bt.off_gs = offs[2];
    bt.off_int = offs[3];
    bt.blocks_main = om[n];
    bt.blocks_prep = op[n];
    bt.blocks_gs = og[n];
    bt.blocks_int = oi[n];
    bt.blocks_marked = std::max(1, std::min(marked, 65535));
    bt.max_tile_threads = max_threads;
    bt.cells_per_thread = cpt;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return bail(fail(LBIB_ECUDA, "querying the device failed"));
        bt.ib_grid_cap = BATCH_IB_BLOCKS_PER_SM * sms;
    }
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&b->ib, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithPriority(&b->cap_ib, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->e_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->e_main, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->e_ib, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(LBIB_ECUDA, "creating batch streams or events failed"));
    b->class_cpt.assign(b->classes.size(), cpt);
    const cudaError_t ce = capture_batch_graph(b);
    if (ce != cudaSuccess)
        return bail(fail(LBIB_ECUDA, std::string("batch graph capture failed: ") + cudaGetErrorString(ce)));
    for (lbib_ctx *c : b->ctx) c->batch = b;
    *out = b;
    return LBIB_OK;
}

int lb_batch_step(lbib_batch *b, long long n) {
    if (!b) return fail(LBIB_EINVAL, "batch is NULL");
    if (n < 0) return fail(LBIB_EINVAL, "n_steps < 0");
    // the graph was captured starting at the creation step's parity
    bool forked = false;
    long long cells = 0;
    for (const lbib_ctx *c : b->ctx) cells += c->L.N;
    const bool graphs = use_graphs(cells);
    while (n > 0) {
        const long long s = b->ctx[0]->step;
        if (graphs && !b->profiling && ((s - b->step) & 1) == 0 && n >= GRAPH_STEPS) {
            if (forked) {
                CU(cudaStreamWaitEvent(b->user, b->e_ib, 0));
                forked = false;
            }
            CU(cudaGraphLaunch(b->graph, b->user));
            for (lbib_ctx *c : b->ctx) c->step += GRAPH_STEPS;
            n -= GRAPH_STEPS;
        } else {
            if (!forked) {
                CU(batch_fork(b, b->user, b->ib));
                forked = true;
            }
            CU(batch_enqueue_step(b, (s & 1) != 0, b->user, b->ib, b->profiling));
            for (lbib_ctx *c : b->ctx) c->step += 1;
            n -= 1;
        }
    }
    if (forked) CU(cudaStreamWaitEvent(b->user, b->e_ib, 0));
    return LBIB_OK;
}

int lb_batch_profile(lbib_batch *b, int on) {
    if (!b) return fail(LBIB_EINVAL, "batch is NULL");
    CU(cudaStreamSynchronize(b->user));
    b->profiling = on != 0;
    b->ev_used = 0;
    return LBIB_OK;
}

int lb_batch_profile_read(lbib_batch *b, double *total_ms, long long *launches) {
    if (!b || !total_ms || !launches) return fail(LBIB_EINVAL, "NULL argument");
    CU(cudaStreamSynchronize(b->user));
    double t = 0.0;
    for (size_t k = 0; k + 1 < b->ev_used; k += 2) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, b->ev[k], b->ev[k + 1]));
        t += ms;
    }
    *total_ms = t;
    *launches = (long long)(b->ev_used / 2);
    return LBIB_OK;
}

int lb_batch_autotune(lbib_batch *b, int steps_per_trial, lbib_batch_tuning *report) {
    if (!b) return fail(LBIB_EINVAL, "batch is NULL");
    if (steps_per_trial < 1) return fail(LBIB_EINVAL, "steps_per_trial < 1");
    const int n_trial = (steps_per_trial + 1) / 2 * 2;
    const bool was_profiling = b->profiling;
    const long long step0 = b->ctx[0]->step;
    const size_t nc = b->classes.size();
    std::vector<std::array<double, 3>> us(nc, std::array<double, 3>{0.0, 0.0, 0.0});
    CU(cudaStreamSynchronize(b->user));
    b->profiling = true;  // kernel by kernel
    b->ev_used = 0;
    // 1. cells per thread of each class's main fluid launch
    const int cands[3] = {1, 2, 4};
    const std::vector<int> best0 = b->class_cpt;
    for (int ci = 0; ci < 3; ++ci) {
        const int cand = cands[ci];
        bool any = false;
        for (size_t k = 0; k < nc; ++k) {
            const bool ok = cpt_valid(b, k, cand);
            b->class_cpt[k] = ok ? cand : best0[k];
            any |= ok;
        }
        if (!any) continue;
        b->class_timing = true;
        b->tev_used = 0;
        const int st = lb_batch_step(b, n_trial);
        b->class_timing = false;
        if (st != LBIB_OK) return st;
        CU(cudaStreamSynchronize(b->user));
        std::vector<double> sum(nc, 0.0);
        std::vector<int> cnt(nc, 0);
        for (size_t e = 0; e + 1 < b->tev_used; e += 2) {
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, b->tev[e], b->tev[e + 1]));
            const int k = b->tev_class[e];
            sum[k] += ms * 1e3;
            cnt[k] += 1;
        }
        for (size_t k = 0; k < nc; ++k)
            if (cpt_valid(b, k, cand) && cnt[k]) us[k][ci] = sum[k] / cnt[k];
    }
    for (size_t k = 0; k < nc; ++k) {
        int best = best0[k];
        double t_best = 1e300;
        for (int ci = 0; ci < 3; ++ci)
            if (us[k][ci] > 0.0 && us[k][ci] < t_best) {
                t_best = us[k][ci];
                best = cands[ci];
            }
        b->class_cpt[k] = best;
    }
    // 2. grid of the marked-tile launch (whole-step timing)
    int mc[4] = {0, 0, 0, 0};
    double mus[4] = {0.0, 0.0, 0.0, 0.0};
    int n_mc = 0;
    if (b->any_nodes) {
        int sms = 0, dev = 0;
        CU(cudaGetDevice(&dev));
        CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int base = b->bt.blocks_marked;
        const int cand_m[4] = {base, std::max(1, base / 2), std::min(65535, 2 * base), std::max(1, 2 * sms)};
        for (int c : cand_m) {
            bool dup = false;
            for (int q = 0; q < n_mc; ++q) dup |= mc[q] == c;
            if (!dup) mc[n_mc++] = c;
        }
        cudaEvent_t t0, t1;
        CU(cudaEventCreate(&t0));
        CU(cudaEventCreate(&t1));
        for (int q = 0; q < n_mc; ++q) {
            b->bt.blocks_marked = mc[q];
            CU(cudaEventRecord(t0, b->user));
            const int st = lb_batch_step(b, n_trial);
            if (st != LBIB_OK) return st;
            CU(cudaEventRecord(t1, b->user));
            CU(cudaEventSynchronize(t1));
            float ms = 0.f;
            CU(cudaEventElapsedTime(&ms, t0, t1));
            mus[q] = ms * 1e3 / n_trial;
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        int qb = 0;
        for (int q = 1; q < n_mc; ++q)
            if (mus[q] < mus[qb]) qb = q;
        b->bt.blocks_marked = mc[qb];
    }
    b->profiling = was_profiling;
    b->ev_used = 0;
    const cudaError_t ce = capture_batch_graph(b);
    if (ce != cudaSuccess) return fail(LBIB_ECUDA, std::string("batch graph capture failed: ") + cudaGetErrorString(ce));
    if (report) {
        memset(report, 0, sizeof(*report));
        report->n_classes = (int)nc;
        for (size_t k = 0; k < nc && k < LBIB_TUNE_MAX_CLASSES; ++k) {
            const DevCtx &c = b->classes[k].box[0];
            report->class_dims[k][0] = c.nx;
            report->class_dims[k][1] = c.ny;
            report->class_dims[k][2] = c.nz;
            report->class_boxes[k] = b->classes[k].n;
            report->class_cells_per_thread[k] = b->class_cpt[k];
            for (int ci = 0; ci < 3; ++ci) report->class_us[k][ci] = us[k][ci];
        }
        for (int q = 0; q < n_mc; ++q) {
            report->marked_candidates[q] = mc[q];
            report->marked_step_us[q] = mus[q];
        }
        report->marked_blocks = b->bt.blocks_marked;
        report->steps_taken = b->ctx[0]->step - step0;
    }
    return LBIB_OK;
}

int lb_batch_destroy(lbib_batch *b) {
    if (!b) return LBIB_OK;
    cudaStreamSynchronize(b->user);
    if (b->ib) cudaStreamSynchronize(b->ib);
    for (lbib_ctx *c : b->ctx)
        if (c && c->batch == b) c->batch = nullptr;
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : b->tev) cudaEventDestroy(e);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->cap_ib) cudaStreamDestroy(b->cap_ib);
    if (b->ib) cudaStreamDestroy(b->ib);
    if (b->e_fork) cudaEventDestroy(b->e_fork);
    if (b->e_main) cudaEventDestroy(b->e_main);
    if (b->e_ib) cudaEventDestroy(b->e_ib);
    if (b->dev) cudaFree(b->dev);
    delete b;
    return LBIB_OK;
}

}  // extern "C"
