// ww_api.cu -- the C ABI declared in include/ww.h: context lifetime, the DtN
// entry points, and the RK4 driver of shoot / shoot_jacobian.  One RK4 step
// (four stages, each: base geometry -> assembly -> factor -> base solve and
// DtN -> base RHS -> variational solves and DtN -> variational RHS) is
// captured once per context into a CUDA graph and replayed `steps` times; in
// the mixed form the base chain runs one stage ahead of the columns on a
// second branch of that graph (capture_overlapped).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "ww_internal.cuh"

namespace ww {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

// twiddles tw[2k], tw[2k+1] = cos, -sin(2 pi k/N) (k < N/2); cs = cos(2 pi m/N),
// sin(2 pi m/N), cot(pi m/N) (m < N; cot slot 0 unused), exact at multiples of pi/2
void fill_tables(int N, double *tw, double *cs) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int k = 0; k < N / 2; ++k) {
        tw[2 * k] = std::cos(two_pi * (double)k / (double)N);
        tw[2 * k + 1] = -std::sin(two_pi * (double)k / (double)N);
    }
    for (int m = 0; m < N; ++m) {
        cs[m] = std::cos(two_pi * (double)m / (double)N);
        cs[N + m] = std::sin(two_pi * (double)m / (double)N);
        cs[2 * N + m] = m == 0 ? 0.0 : 1.0 / std::tan(0.5 * two_pi * (double)m / (double)N);
    }
    for (int m = 0; m < N; m += N / 4) {
        int q = m / (N / 4);
        cs[m] = (q == 0) ? 1.0 : (q == 2 ? -1.0 : 0.0);
        cs[N + m] = (q == 1) ? 1.0 : (q == 3 ? -1.0 : 0.0);
        if (q == 2) cs[2 * N + m] = 0.0;
    }
    for (int k = 0; k < N / 2; k += N / 4) {
        int q = k / (N / 4);
        tw[2 * k] = q == 0 ? 1.0 : 0.0;
        tw[2 * k + 1] = q == 0 ? 0.0 : -1.0;
    }
}

namespace {

constexpr int NPH = WW_NPHASE;
constexpr int EV_PER_STEP = 4 * NPH * 2;   // [stage][phase][begin/end]

struct StepGraph {
    cudaGraph_t graph = nullptr;              // kept alive: its event nodes are re-pointed per replay
    cudaGraphExec_t exec = nullptr;
    std::vector<std::pair<cudaGraphNode_t, int>> ev_nodes;   // node -> flat event slot
    int nkern = 0;                            // kernel nodes (launches per replay)
    unsigned marked[4] = {};                  // per stage: phases with event nodes in this program
};

int count_kernel_nodes(cudaGraph_t g, int *out) {
    size_t nn = 0;
    WW_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    WW_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &nn));
    int k = 0;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        WW_CUDA_TRY(cudaGraphNodeGetType(nd, &t));
        if (t == cudaGraphNodeTypeKernel) ++k;
    }
    *out = k;
    return WW_OK;
}

struct Owned {
    Ctx c;
    double *cbuf = nullptr, *rbuf = nullptr, *Jbuf = nullptr, *fbuf = nullptr;
    StepGraph graphs[2][2];                   // [with_columns][timing]
    StepGraph prologue[2];                    // [with_columns]: initial data (+ the mixed inverse)
    cudaStream_t own_stream = nullptr;        // created by ww_create, used unless ww_set_stream overrides
    cudaStream_t side_stream = nullptr;       // the base chain's branch inside captured step graphs
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_base[4] = {}, ev_cols[4] = {};   // capture fork/join
    std::vector<void *> allocs;
    // phase timing
    bool timing = false;
    bool capturing = false;
    bool in_shot = false;                     // the stages of a shot are being issued (marks allowed)
    int replay = 0;                           // RK step being launched
    unsigned marked[4] = {};                  // per stage: phases recorded by the current step program
    cudaEvent_t placeholder[EV_PER_STEP] = {};
    std::vector<cudaEvent_t> pool;            // steps * EV_PER_STEP
    double ph_ms[NPH] = {};
    int ph_count[NPH] = {};
    // the adjoint sweep (allocated by its first call): trajectory records and
    // the forward step, the turn-around and the backward step as graphs
    AdjWs adj = {};
    StepGraph adj_fwd, adj_mid, adj_bwd;
    StepGraph adj_restart, adj_reentry;       // checkpointed sweep: segment restart (forward) and re-entry (backward)
    // the batch graph: this shot's step counter, and identifiers that key cached batch graphs
    int *loop_count = nullptr;
    unsigned long long id = 0;                // unique per context, never reused
    unsigned long long version = 0;           // bumped whenever the captured step programs are dropped
};

void destroy_graph(StepGraph &sg) {
    if (sg.exec) cudaGraphExecDestroy(sg.exec);
    if (sg.graph) cudaGraphDestroy(sg.graph);
    sg = StepGraph();
}

void drop_batch_graphs(unsigned long long id);   // below

// every captured program of a context (after a change of its schedule or verification)
void drop_graphs(Owned *o) {
    for (int w = 0; w < 2; ++w) {
        for (int t = 0; t < 2; ++t) destroy_graph(o->graphs[w][t]);
        destroy_graph(o->prologue[w]);
    }
    for (StepGraph *sg : {&o->adj_fwd, &o->adj_mid, &o->adj_bwd, &o->adj_restart, &o->adj_reentry}) destroy_graph(*sg);
    o->version += 1;
    drop_batch_graphs(o->id);
}

// record the begin (b = 0) or end (b = 1) event of a phase of stage st
int mark(Ctx *c, int st, int phase, int b) {
    Owned *o = reinterpret_cast<Owned *>(c->owner);
    if (!o || !o->timing || !o->in_shot) return WW_OK;
    o->marked[st & 3] |= 1u << phase;
    const int slot = (st * NPH + phase) * 2 + b;
    if (o->capturing) {
        // an "external" record becomes an event-record node of the captured graph
        WW_CUDA_TRY(cudaEventRecordWithFlags(o->placeholder[slot], c->stream, cudaEventRecordExternal));
    } else {
        WW_CUDA_TRY(cudaEventRecord(o->pool[(size_t)o->replay * EV_PER_STEP + slot], c->stream));
    }
    return WW_OK;
}

int dalloc(Owned *o, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return fail(WW_ERR_ALLOC, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    o->allocs.push_back(*p);
    o->c.dev_bytes += bytes;
    return WW_OK;
}

void dfree(Owned *o, void *p) {
    if (!p) return;
    for (size_t i = 0; i < o->allocs.size(); ++i)
        if (o->allocs[i] == p) {
            o->allocs.erase(o->allocs.begin() + (long)i);
            break;
        }
    cudaFree(p);
}

template <typename T>
int dalloc_n(Owned *o, T **p, size_t n) {
    return dalloc(o, reinterpret_cast<void **>(p), sizeof(T) * (n ? n : 1));
}

Owned *owner(ww_ctx *ctx) { return reinterpret_cast<Owned *>(ctx); }

// fresh: start the mixed inverse from scratch; update: move it to this stage's A
int factor(Ctx *c, int fresh = 0, int update = 1) {
    if (c->precision == WW_MIXED) return mixed_setup(c, fresh, update);
    return lu_factor_fp64(c);
}

int solve(Ctx *c, double *B, int ncols) {
    if (c->precision == WW_MIXED) return mixed_solve(c, B, ncols);
    return lu_solve_fp64(c, B, ncols);
}

// Gout[:, col0 : col0+ncols] += G Gam[:, col0 : ...]; st >= 0 times the product kernel
int apply_G(Ctx *c, int col0, int ncols, int st = -1) {
    if (c->precision == WW_MIXED) {
        WW_TRY(mixed_apply_G(c, col0, ncols, 0));                 // operand split (none when narrow)
        if (st >= 0) WW_TRY(mark(c, st, WW_PHASE_GKERNEL, 0));
        WW_TRY(mixed_apply_G(c, col0, ncols, 1));                 // the product
        if (st >= 0) WW_TRY(mark(c, st, WW_PHASE_GKERNEL, 1));
        return WW_OK;
    }
    if (st >= 0) WW_TRY(mark(c, st, WW_PHASE_GKERNEL, 0));
    WW_TRY(dgemm(c->stream, c->N, ncols, c->N, 1.0, c->G, c->N, c->Gam + (size_t)col0 * c->N, c->N, 1.0,
                 c->Gout + (size_t)col0 * c->N, c->N));
    if (st >= 0) WW_TRY(mark(c, st, WW_PHASE_GKERNEL, 1));
    return WW_OK;
}

// The base chain of RK stage st: geometry, DtN setup (assembly, factor / inverse
// update and the per-stage operands) and the base state's own DtN and right-hand
// side with its RK update.  It reads and writes only the base column of the
// state, so it does not depend on the variational columns.
// ns_every: move the mixed inverse to every stage's A (when the base chain is
// hidden behind the columns: a fresher inverse saves column refinement
// iterations), else on even stages and on odd ones only when it drifted.
int run_base(Ctx *c, int st, const double *cvec, bool ns_every = false) {
    c->cur_stage = st;
    WW_TRY(launch_base_geometry(c, c->Ys, c->Ys + c->N, 1));
    WW_TRY(mark(c, st, WW_PHASE_ASSEMBLY, 0));
    WW_TRY(launch_assemble(c));
    WW_TRY(mark(c, st, WW_PHASE_ASSEMBLY, 1));
    WW_TRY(mark(c, st, WW_PHASE_FACTOR, 0));
    WW_TRY(factor(c, 0, ns_every || (st % 2) == 0));
    WW_TRY(mark(c, st, WW_PHASE_FACTOR, 1));
    WW_TRY(mark(c, st, WW_PHASE_BASE, 0));
    WW_TRY(launch_phi0(c));
    WW_TRY(solve(c, c->M, 1));
    WW_TRY(launch_gamma(c, 0, 1));
    WW_TRY(apply_G(c, 0, 1));
    WW_TRY(launch_base_rhs(c, st, cvec));
    WW_TRY(mark(c, st, WW_PHASE_BASE, 1));
    return WW_OK;
}

// The variational columns of RK stage st (App. B): they read the base results
// of the same stage (its DtN operands, u, v, w3 and F).
int run_cols(Ctx *c, int st, const double *cvec) {
    if (c->nc <= 0) return WW_OK;
    c->cur_stage = st;
    WW_TRY(launch_psi(c));
    WW_TRY(mark(c, st, WW_PHASE_SOLVE, 0));
    WW_TRY(solve(c, c->M + c->N, c->nc));
    WW_TRY(mark(c, st, WW_PHASE_SOLVE, 1));
    WW_TRY(mark(c, st, WW_PHASE_GAMMA, 0));
    WW_TRY(launch_gamma(c, 1, c->nc));
    WW_TRY(mark(c, st, WW_PHASE_GAMMA, 1));
    WW_TRY(mark(c, st, WW_PHASE_GAPPLY, 0));
    WW_TRY(apply_G(c, 1, c->nc, st));
    WW_TRY(mark(c, st, WW_PHASE_GAPPLY, 1));
    WW_TRY(mark(c, st, WW_PHASE_COLRHS, 0));
    WW_TRY(launch_col_rhs(c, st, cvec));
    WW_TRY(mark(c, st, WW_PHASE_COLRHS, 1));
    return WW_OK;
}

// one RK4 stage in order; cvec is the context's device copy of c (T = cvec[0])
int run_stage(Ctx *c, int st, const double *cvec, int with_cols) {
    select_parity(c, st & 1);
    WW_TRY(run_base(c, st, cvec));
    if (with_cols) WW_TRY(run_cols(c, st, cvec));
    return WW_OK;
}

// In the mixed form a Jacobian step runs as two chains: the base chain one
// stage ahead on a second stream, the column chain of the stage before on the
// caller's stream (the column work is tensor-core bound, the base chain is
// mostly latency bound, so they share the GPU well).  Per-stage buffers
// alternate by stage parity.  One replay covers
//   columns of stages 0..3 of this step  ||  base of stages 1..3 and of stage 0 of the next step,
// with  columns(s) after base(s)  and  base(s+1) after columns(s-1)  (the
// latter frees the parity buffers base(s+1) overwrites).  Before the first
// replay the prologue runs base(0); the last replay's base(0) is for a step
// that is not taken and changes nothing that is read afterwards.
bool overlapped(const Owned *o, int with_cols) {
    const Ctx *c = &o->c;
    return c->precision == WW_MIXED && with_cols && c->nc > 0 && c->stream != nullptr && o->side_stream != nullptr &&
           c->sch.overlap != 0;
}

int capture_overlapped(Owned *o, const double *cvec) {
    Ctx *c = &o->c;
    cudaStream_t main_s = c->stream, side = o->side_stream;
    int st = WW_OK;
    WW_CUDA_TRY(cudaEventRecord(o->ev_fork, main_s));
    WW_CUDA_TRY(cudaStreamWaitEvent(side, o->ev_fork, 0));
    for (int s = 0; s < 4 && st == WW_OK; ++s) {
        c->stream = main_s;
        if (s > 0) WW_CUDA_TRY(cudaStreamWaitEvent(main_s, o->ev_base[s], 0));
        select_parity(c, s & 1);
        st = run_cols(c, s, cvec);
        if (st != WW_OK) break;
        WW_CUDA_TRY(cudaEventRecord(o->ev_cols[s], main_s));
        c->stream = side;
        if (s > 0) {
            cudaError_t e = cudaStreamWaitEvent(side, o->ev_cols[s - 1], 0);
            if (e != cudaSuccess) st = fail(WW_ERR_CUDA, std::string("capture join: ") + cudaGetErrorString(e));
        }
        select_parity(c, (s + 1) & 1);
        if (st == WW_OK) st = run_base(c, (s + 1) & 3, cvec, c->sch.ns_every == 1);
        if (st == WW_OK && s < 3) {
            cudaError_t e = cudaEventRecord(o->ev_base[s + 1], side);
            if (e != cudaSuccess) st = fail(WW_ERR_CUDA, std::string("capture fork: ") + cudaGetErrorString(e));
        }
    }
    c->stream = main_s;
    select_parity(c, 0);
    if (st != WW_OK) return st;
    WW_CUDA_TRY(cudaEventRecord(o->ev_join, side));
    WW_CUDA_TRY(cudaStreamWaitEvent(main_s, o->ev_join, 0));
    return WW_OK;
}

int build_step_graph(Owned *o, int with_cols) {
    Ctx *c = &o->c;
    StepGraph &sg = o->graphs[with_cols][o->timing ? 1 : 0];
    if (sg.exec) return WW_OK;
    cudaGraph_t g = nullptr;
    WW_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    o->capturing = true;
    for (unsigned &m : o->marked) m = 0;
    int st = WW_OK;
    if (overlapped(o, with_cols))
        st = capture_overlapped(o, o->cbuf);
    else
        for (int s = 0; s < 4 && st == WW_OK; ++s) st = run_stage(c, s, o->cbuf, with_cols);
    o->capturing = false;
    for (int k = 0; k < 4; ++k) sg.marked[k] = o->marked[k];
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != WW_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(WW_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    if (o->timing) {
        // find the event-record nodes and map each to its [stage][phase][b] slot
        size_t nn = 0;
        WW_CUDA_TRY(cudaGraphGetNodes(g, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        WW_CUDA_TRY(cudaGraphGetNodes(g, nodes.data(), &nn));
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            WW_CUDA_TRY(cudaGraphNodeGetType(nd, &t));
            if (t != cudaGraphNodeTypeEventRecord) continue;
            cudaEvent_t ev;
            WW_CUDA_TRY(cudaGraphEventRecordNodeGetEvent(nd, &ev));
            for (int k = 0; k < EV_PER_STEP; ++k)
                if (o->placeholder[k] == ev) sg.ev_nodes.emplace_back(nd, k);
        }
        if (sg.ev_nodes.empty()) {
            cudaGraphDestroy(g);
            return fail(WW_ERR_CUDA, "phase timing: no event-record nodes in the captured step");
        }
    }
    WW_TRY(count_kernel_nodes(g, &sg.nkern));
    // prio: the kernel nodes keep the priorities of the streams they were
    // captured on (the base chain's side stream is the device's highest)
    e = cudaGraphInstantiate(&sg.exec, g, c->sch.prio ? cudaGraphInstantiateFlagUseNodePriority : 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(WW_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    sg.graph = g;
    return WW_OK;
}

// initial data (and, in WW_MIXED, the approximate inverse of the initial
// surface): one graph per context, replayed at the start of every shot
int prologue(Owned *o, const double *cvec, int with_cols) {
    Ctx *c = &o->c;
    select_parity(c, 0);
    WW_TRY(launch_initial(c, cvec, with_cols));
    if (c->precision == WW_MIXED) {
        WW_TRY(launch_base_geometry(c, c->Ys, c->Ys + c->N, 1));
        WW_TRY(launch_assemble(c));
        WW_TRY(factor(c, 1));
        if (overlapped(o, with_cols))   // the base chain runs one stage ahead
            WW_TRY(run_base(c, 0, cvec, c->sch.ns_every == 1));
    }
    return WW_OK;
}

int build_prologue_graph(Owned *o, int with_cols);

int run_prologue(Owned *o, int with_cols) {
    Ctx *c = &o->c;
    if (c->stream == nullptr) {
        const bool timing = o->timing;
        o->timing = false;   // the prologue is not part of the timed phases
        const int st = prologue(o, o->cbuf, with_cols);
        o->timing = timing;
        return st;
    }
    WW_TRY(build_prologue_graph(o, with_cols));
    WW_CUDA_TRY(cudaGraphLaunch(o->prologue[with_cols].exec, c->stream));
    return WW_OK;
}

int build_prologue_graph(Owned *o, int with_cols) {
    Ctx *c = &o->c;
    const bool timing = o->timing;
    o->timing = false;   // the prologue is not part of the timed phases
    int st = WW_OK;
    StepGraph &pg = o->prologue[with_cols];
    if (!pg.exec) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            o->timing = timing;
            return fail(WW_ERR_CUDA, std::string("prologue capture: ") + cudaGetErrorString(e));
        }
        st = prologue(o, o->cbuf, with_cols);
        e = cudaStreamEndCapture(c->stream, &g);
        o->timing = timing;
        if (st != WW_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail(WW_ERR_CUDA, std::string("prologue capture: ") + cudaGetErrorString(e));
        WW_TRY(count_kernel_nodes(g, &pg.nkern));
        e = cudaGraphInstantiate(&pg.exec, g, 0);
        pg.graph = g;
        if (e != cudaSuccess) return fail(WW_ERR_CUDA, std::string("prologue instantiate: ") + cudaGetErrorString(e));
    }
    o->timing = timing;
    return WW_OK;
}

int ensure_timing_events(Owned *o) {
    const size_t need = (size_t)o->c.steps * EV_PER_STEP;
    if (!o->placeholder[0])
        for (int k = 0; k < EV_PER_STEP; ++k) WW_CUDA_TRY(cudaEventCreate(&o->placeholder[k]));
    while (o->pool.size() < need) {
        cudaEvent_t ev;
        WW_CUDA_TRY(cudaEventCreate(&ev));
        o->pool.push_back(ev);
    }
    return WW_OK;
}

int collect_timing(Owned *o) {
    for (int p = 0; p < NPH; ++p) {
        o->ph_ms[p] = 0.0;
        o->ph_count[p] = 0;
    }
    for (int rep = 0; rep < o->c.steps; ++rep)
        for (int st = 0; st < 4; ++st)
            for (int p = 0; p < NPH; ++p) {
                if (!(o->marked[st] & (1u << p))) continue;   // a phase this stage does not run
                const size_t base = (size_t)rep * EV_PER_STEP + (size_t)(st * NPH + p) * 2;
                float ms = 0.f;
                WW_CUDA_TRY(cudaEventElapsedTime(&ms, o->pool[base], o->pool[base + 1]));
                o->ph_ms[p] += ms;
                o->ph_count[p] += 1;
            }
    return WW_OK;
}

int check_status(Ctx *c) {
    int st = 0;
    WW_CUDA_TRY(cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (c->precision == WW_MIXED) {
        double ratio = 0, nsres = 0, vmax = 0;
        int err = 0, iters[3] = {0, 0, 0}, vn = 0;
        WW_TRY(mixed_read_stats(c, &ratio, &nsres, iters, &err, &vmax, &vn));
        c->stats.refine_resid_max = ratio;
        c->stats.refine_resid_measured = vn > 0 ? vmax : -1.0;
        c->stats.verified_solves = vn;
        c->stats.ns_resid_max = nsres;
        c->stats.refine_iters_max = iters[0];
        c->stats.refine_iters_mean = iters[2] > 0 ? (double)iters[1] / iters[2] : 0.0;
        if (err) return fail(WW_ERR_TIMEOUT, "a tensor-core kernel gave up waiting (bounded wait expired)");
    }
    if (st & ST_NO_CONV)
        return fail(WW_ERR_NO_CONVERGENCE, "iterative refinement missed its tolerance (or the approximate inverse "
                                           "lost contact: the surface moved too far in one RK stage)");
    if (st & ST_GEOMETRY)
        return fail(WW_ERR_GEOMETRY, "surface touches the bottom (finite depth needs eta > 0) or is non-finite");
    if (st & ST_NONFINITE)
        return fail(WW_ERR_GEOMETRY, "non-finite value in a right-hand side or factor (is dt within RK4 stability?)");
    return WW_OK;
}

int run_shot(Owned *o, const double *cvec, bool c_on_host, double *r, double *J, double *f, int with_cols) {
    Ctx *c = &o->c;
    c->one_col = !with_cols;   // (graphs are captured per with_cols, each with its own setting)
    WW_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    WW_CUDA_TRY(cudaMemcpyAsync(o->cbuf, cvec, sizeof(double) * (c->n + 1),
                                c_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    WW_TRY(run_prologue(o, with_cols));
    if (o->timing) WW_TRY(ensure_timing_events(o));
    for (unsigned &m : o->marked) m = 0;
    struct InShot {
        Owned *o;
        InShot(Owned *o_) : o(o_) { o->in_shot = true; }
        ~InShot() { o->in_shot = false; }
    } in_shot(o);
    if (c->stream == nullptr) {
        // the legacy default stream cannot be captured: launch the stages directly
        for (int s = 0; s < c->steps; ++s) {
            o->replay = s;
            for (int k = 0; k < 4; ++k) WW_TRY(run_stage(c, k, o->cbuf, with_cols));
        }
    } else {
        WW_TRY(build_step_graph(o, with_cols));
        StepGraph &sg = o->graphs[with_cols][o->timing ? 1 : 0];
        for (int k = 0; k < 4; ++k) o->marked[k] = sg.marked[k];
        for (int s = 0; s < c->steps; ++s) {
            if (o->timing)
                for (auto &ne : sg.ev_nodes)
                    WW_CUDA_TRY(cudaGraphExecEventRecordNodeSetEvent(
                        sg.exec, ne.first, o->pool[(size_t)s * EV_PER_STEP + ne.second]));
            WW_CUDA_TRY(cudaGraphLaunch(sg.exec, c->stream));
        }
    }
    WW_TRY(launch_outputs(c, r, J, f, with_cols));
    c->stats.stages = 4 * c->steps;
    c->stats.device_bytes = (long long)c->dev_bytes;
    c->stats.adjoint_bytes = (long long)o->adj.bytes;
    if (c->stream == nullptr)
        c->stats.launches = -1;   // direct launches are not counted
    else
        c->stats.launches = (long long)o->prologue[with_cols].nkern +
                            (long long)c->steps * o->graphs[with_cols][o->timing ? 1 : 0].nkern + (with_cols ? 2 : 1);
    c->dtn_ready = false;   // the operator now belongs to the last stage's surface
    WW_TRY(check_status(c));
    if (o->timing) WW_TRY(collect_timing(o));
    return WW_OK;
}

// ---------------------------------------------------------------- discrete adjoint
// steps of records held: all of them, or the checkpoint interval
int held_steps(const Ctx *c) { return c->ckpt_every > 0 && c->ckpt_every < c->steps ? c->ckpt_every : c->steps; }

void free_adjoint(Owned *o) {
    AdjWs &a = o->adj;
    for (void *p : {(void *)a.rec, (void *)a.lam, (void *)a.kb, (void *)a.eta, (void *)a.chi, (void *)a.y,
                    (void *)a.etal, (void *)a.psil, (void *)a.gT, (void *)a.step, (void *)a.A2, (void *)a.G2,
                    (void *)a.X2, (void *)a.ckpt})
        dfree(o, p);
    o->c.dev_bytes -= a.bytes;
    a = AdjWs{};
    for (StepGraph *sg : {&o->adj_fwd, &o->adj_mid, &o->adj_bwd, &o->adj_restart, &o->adj_reentry}) {
        if (sg->exec) cudaGraphExecDestroy(sg->exec);
        if (sg->graph) cudaGraphDestroy(sg->graph);
        *sg = StepGraph();
    }
}

int ensure_adjoint(Owned *o) {
    AdjWs &a = o->adj;
    const Ctx *c = &o->c;
    const int K = held_steps(c);
    if (a.rec && a.kheld == K) return WW_OK;
    if (a.rec) free_adjoint(o);   // the checkpoint interval changed: the record buffer's size with it
    const size_t N = (size_t)c->N, before = o->c.dev_bytes;
    WW_TRY(dalloc_n(o, &a.rec, (size_t)4 * K * ADJ_REC * N));
    a.kheld = K;
    if (K < c->steps) WW_TRY(dalloc_n(o, &a.ckpt, (size_t)((c->steps + K - 1) / K) * 2 * N));
    WW_TRY(dalloc_n(o, &a.lam, 2 * N));
    WW_TRY(dalloc_n(o, &a.kb, 8 * N));
    WW_TRY(dalloc_n(o, &a.eta, N));
    WW_TRY(dalloc_n(o, &a.chi, N));
    WW_TRY(dalloc_n(o, &a.y, N));
    WW_TRY(dalloc_n(o, &a.etal, N));
    WW_TRY(dalloc_n(o, &a.psil, N));
    WW_TRY(dalloc_n(o, &a.gT, 1));
    WW_TRY(dalloc_n(o, &a.step, 1));
    if (c->precision == WW_MIXED) {   // the overlapped sweep's second operand copies
        WW_TRY(dalloc_n(o, &a.A2, N * N));
        WW_TRY(dalloc_n(o, &a.G2, N * N));
        WW_TRY(dalloc_n(o, &a.X2, N * N));
    }
    a.bytes = o->c.dev_bytes - before;
    return prepare_adjoint(c->N);
}

// The backward sweep's two chains (MIXED on a stream of its own): the DtN setup
// of a stage (its surface, geometry, A^T and G^T, the inverse update) needs
// only the recorded trajectory, not the adjoint vector, so it runs one stage
// ahead on the side stream while the adjoint of the stage before runs on the
// caller's.  A^T, G^T and the FP32 inverse alternate between two copies by
// stage parity; the setup of stage k waits for the adjoint of stage k + 2
// (the last reader of that copy).
bool adj_overlapped(const Owned *o) {
    const Ctx *c = &o->c;
    return c->precision == WW_MIXED && c->stream != nullptr && o->side_stream != nullptr && o->adj.A2 != nullptr;
}

struct AdjOperands {
    double *A[2], *G[2];
    float *X[2];
};

void adj_select(Owned *o, const AdjOperands &ops, int p) {
    Ctx *c = &o->c;
    c->A = ops.A[p];
    c->G = ops.G[p];
    mixed_set_inverse(c, ops.X[p]);
}

// DtN setup of the stage whose record is 4 step + off, into operand copy p
int adj_setup(Owned *o, const AdjOperands &ops, int off, int p, bool fresh) {
    Ctx *c = &o->c;
    adj_select(o, ops, p);
    WW_TRY(launch_adj_fetch(c, &o->adj, off));
    WW_TRY(launch_base_geometry(c, o->adj.eta, o->adj.eta, 0));
    WW_TRY(launch_assemble(c));                  // A^T, G^T
    return factor(c, fresh ? 1 : 0, 1);
}

// the adjoint of stage k of the current step, reading operand copy k & 1
int adj_stage(Owned *o, const AdjOperands &ops, int k) {
    Ctx *c = &o->c;
    AdjWs *a = &o->adj;
    adj_select(o, ops, k & 1);
    WW_TRY(launch_adj_local(c, a, k, o->cbuf));
    WW_TRY(gemv_narrow(c->stream, c->N, 1, c->N, 1.0, c->G, c->N, a->chi, c->N, 0.0, a->y, c->N));   // G^T chi
    WW_TRY(launch_adj_dtn(c, a));
    WW_TRY(solve(c, c->M, 1));                   // A^{-T} D (1/2 H chi - G^T chi)
    return launch_adj_update(c, a, k, o->cbuf);
}

// turn-around of the overlapped sweep: lambda, and the setup of the last stage
// (record 4 steps - 1) with a fresh inverse
int adj_turnaround_overlapped(Owned *o, const AdjOperands &ops) {
    Ctx *c = &o->c;
    select_parity(c, 0);
    WW_TRY(launch_adj_init(c, &o->adj));        // step = steps
    return adj_setup(o, ops, -1, 1, true);
}

// one backward step: adjoints of stages 3..0 on the caller's stream, setups of
// stages 2..0 and of stage 3 of the step before on the side stream
int adj_backward_step_overlapped(Owned *o, const AdjOperands &ops) {
    Ctx *c = &o->c;
    cudaStream_t main_s = c->stream, side = o->side_stream;
    select_parity(c, 0);
    int st = launch_adj_begin_step(c, &o->adj, o->cbuf);   // step -= 1
    if (st != WW_OK) return st;
    WW_CUDA_TRY(cudaEventRecord(o->ev_fork, main_s));
    WW_CUDA_TRY(cudaStreamWaitEvent(side, o->ev_fork, 0));
    for (int k = 3; k >= 0 && st == WW_OK; --k) {
        // side: the setup of the next stage in backward order (k - 1, or stage 3 of the step
        // before), after the adjoint of stage k + 1 released that operand copy
        c->stream = side;
        if (k <= 2) WW_CUDA_TRY(cudaStreamWaitEvent(side, o->ev_cols[k + 1], 0));
        st = adj_setup(o, ops, k - 1, (k - 1) & 1, false);
        if (st != WW_OK) break;
        WW_CUDA_TRY(cudaEventRecord(k > 0 ? o->ev_base[k - 1] : o->ev_join, side));
        // main: the adjoint of stage k (its setup ran in the step before when k = 3)
        c->stream = main_s;
        if (k <= 2) WW_CUDA_TRY(cudaStreamWaitEvent(main_s, o->ev_base[k], 0));
        st = adj_stage(o, ops, k);
        if (st != WW_OK) break;
        WW_CUDA_TRY(cudaEventRecord(o->ev_cols[k], main_s));
    }
    c->stream = main_s;
    if (st != WW_OK) return st;
    WW_CUDA_TRY(cudaStreamWaitEvent(main_s, o->ev_join, 0));
    return WW_OK;
}

// forward: one RK step of the base state, each stage recorded (its surface
// before the stage, its phi_x, phi_y, w3 and F after)
int adj_forward_step(Owned *o) {
    Ctx *c = &o->c;
    for (int k = 0; k < 4; ++k) {
        select_parity(c, k & 1);
        WW_TRY(launch_adj_record_eta(c, &o->adj, k));
        WW_TRY(run_base(c, k, o->cbuf));
        WW_TRY(launch_adj_record_fields(c, &o->adj, k));
    }
    return WW_OK;
}

// turn-around: lambda = (0, phi(T/4)/N), and (mixed form) a fresh inverse of
// the transposed operator at the final surface for the first backward stage
int adj_turnaround(Owned *o) {
    Ctx *c = &o->c;
    select_parity(c, 0);
    WW_TRY(launch_adj_init(c, &o->adj));
    if (c->precision == WW_MIXED) {
        WW_TRY(launch_base_geometry(c, c->Ys, c->Ys, 0));
        WW_TRY(launch_assemble(c));
        WW_TRY(factor(c, 1));
    }
    return WW_OK;
}

// backward: the transposed RK step (filter, then stages 3..0)
int adj_backward_step(Owned *o) {
    Ctx *c = &o->c;
    AdjWs *a = &o->adj;
    select_parity(c, 0);
    WW_TRY(launch_adj_begin_step(c, a, o->cbuf));
    for (int k = 3; k >= 0; --k) {
        WW_TRY(launch_adj_fetch(c, a, k));
        WW_TRY(launch_base_geometry(c, a->eta, a->eta, 0));
        WW_TRY(launch_assemble(c));                  // A^T, G^T
        WW_TRY(factor(c, 0, 1));
        WW_TRY(launch_adj_local(c, a, k, o->cbuf));
        WW_TRY(gemv_narrow(c->stream, c->N, 1, c->N, 1.0, c->G, c->N, a->chi, c->N, 0.0, a->y, c->N));   // G^T chi
        WW_TRY(launch_adj_dtn(c, a));
        WW_TRY(solve(c, c->M, 1));                   // A^{-T} D (1/2 H chi - G^T chi)
        WW_TRY(launch_adj_update(c, a, k, o->cbuf));
    }
    return WW_OK;
}

// run `body` once on the stream, through a graph captured on first use
template <class F>
int replay(Owned *o, StepGraph &sg, F body) {
    Ctx *c = &o->c;
    if (c->stream == nullptr) return body();
    if (!sg.exec) {
        cudaGraph_t g = nullptr;
        WW_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        o->capturing = true;
        const int st = body();
        o->capturing = false;
        const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (st != WW_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail(WW_ERR_CUDA, std::string("adjoint capture: ") + cudaGetErrorString(e));
        WW_TRY(count_kernel_nodes(g, &sg.nkern));
        const cudaError_t ei = cudaGraphInstantiate(&sg.exec, g, 0);
        sg.graph = g;
        if (ei != cudaSuccess) return fail(WW_ERR_CUDA, std::string("adjoint instantiate: ") + cudaGetErrorString(ei));
    }
    WW_CUDA_TRY(cudaGraphLaunch(sg.exec, c->stream));
    return WW_OK;
}

// Checkpointed sweep, restart of a segment from its checkpoint: the base state
// is already in Y and Ys; the mixed form builds a fresh approximate inverse of
// the (forward) operator at that surface, as the prologue does at t = 0.
int adj_restart(Owned *o) {
    Ctx *c = &o->c;
    select_parity(c, 0);
    if (c->precision != WW_MIXED) return WW_OK;
    WW_TRY(launch_base_geometry(c, c->Ys, c->Ys + c->N, 1));
    WW_TRY(launch_assemble(c));
    return factor(c, 1);
}

// Checkpointed sweep, re-entry into the backward steps after a segment was
// recomputed: the mixed form's fresh inverse of the transposed operator at the
// segment's end (the turnaround without lambda), into operand copy 1 in the
// overlapped sweep (where the setup of the segment's last stage goes).
int adj_reentry(Owned *o, const AdjOperands *ops) {
    Ctx *c = &o->c;
    select_parity(c, 0);
    if (ops) return adj_setup(o, *ops, -1, 1, true);
    if (c->precision != WW_MIXED) return WW_OK;
    WW_TRY(launch_base_geometry(c, c->Ys, c->Ys, 0));
    WW_TRY(launch_assemble(c));
    return factor(c, 1);
}

int run_adjoint(Owned *o, const double *cvec, bool c_on_host, double *f, double *grad) {
    Ctx *c = &o->c;
    WW_TRY(ensure_adjoint(o));
    const bool timing = o->timing;
    o->timing = false;   // the phase timers cover the forward Jacobian only
    const bool ovl = adj_overlapped(o);
    // operand copy 0 is the context's own A, G, X; copy 1 the sweep's second set
    const AdjOperands ops{{c->A, o->adj.A2}, {c->G, o->adj.G2}, {c->mx ? mixed_set_inverse(c, nullptr) : nullptr,
                                                                 o->adj.X2}};
    struct Restore {
        Owned *o;
        bool t;
        const AdjOperands *ops;
        ~Restore() {
            o->timing = t;
            o->c.trans = 0;
            if (ops) adj_select(o, *ops, 0);
        }
    } restore{o, timing, ovl ? &ops : nullptr};
    c->one_col = true;
    const size_t N = (size_t)c->N;
    const int K = held_steps(c);                       // steps per segment
    const int nseg = (c->steps + K - 1) / K;
    WW_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    WW_CUDA_TRY(cudaMemsetAsync(o->adj.step, 0, sizeof(int), c->stream));
    WW_CUDA_TRY(cudaMemcpyAsync(o->cbuf, cvec, sizeof(double) * (c->n + 1),
                                c_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream));
    c->trans = 0;
    WW_TRY(run_prologue(o, 0));
    // forward: the base trajectory, each stage recorded into the segment's
    // slots; in checkpointed mode the state at each segment start is kept and
    // the record counter restarts there
    for (int s = 0; s < c->steps; ++s) {
        if (K < c->steps && s % K == 0) {
            WW_CUDA_TRY(cudaMemcpyAsync(o->adj.ckpt + (size_t)(s / K) * 2 * N, c->Y, sizeof(double) * 2 * N,
                                        cudaMemcpyDeviceToDevice, c->stream));
            WW_TRY(launch_adj_set_step(c, &o->adj, 0));
        }
        WW_TRY(replay(o, o->adj_fwd, [&] { return adj_forward_step(o); }));
    }
    WW_TRY(launch_outputs(c, o->rbuf, nullptr, f, 0));
    long long launches = (long long)o->prologue[0].nkern + (long long)c->steps * o->adj_fwd.nkern + 1 +
                         (K < c->steps ? nseg : 0);
    // backward, segment by segment from the last; the last segment's records
    // are those of the forward pass
    c->trans = 1;
    if (ovl)
        WW_TRY(replay(o, o->adj_mid, [&] { return adj_turnaround_overlapped(o, ops); }));
    else
        WW_TRY(replay(o, o->adj_mid, [&] { return adj_turnaround(o); }));
    launches += o->adj_mid.nkern;
    for (int j = nseg - 1; j >= 0; --j) {
        const int L = j == nseg - 1 ? c->steps - j * K : K;
        if (j < nseg - 1) {
            // recompute the segment's records from its checkpoint
            if (ovl) adj_select(o, ops, 0);
            c->trans = 0;
            const double *ck = o->adj.ckpt + (size_t)j * 2 * N;
            WW_CUDA_TRY(cudaMemcpyAsync(c->Y, ck, sizeof(double) * 2 * N, cudaMemcpyDeviceToDevice, c->stream));
            WW_CUDA_TRY(cudaMemcpyAsync(c->Ys, ck, sizeof(double) * 2 * N, cudaMemcpyDeviceToDevice, c->stream));
            WW_TRY(launch_adj_set_step(c, &o->adj, 0));
            WW_TRY(replay(o, o->adj_restart, [&] { return adj_restart(o); }));
            for (int s = 0; s < L; ++s) WW_TRY(replay(o, o->adj_fwd, [&] { return adj_forward_step(o); }));
            c->trans = 1;
            WW_TRY(replay(o, o->adj_reentry, [&] { return adj_reentry(o, ovl ? &ops : nullptr); }));
            launches += 1 + o->adj_restart.nkern + (long long)L * o->adj_fwd.nkern + o->adj_reentry.nkern;
        }
        for (int s = 0; s < L; ++s) {
            if (ovl)
                WW_TRY(replay(o, o->adj_bwd, [&] { return adj_backward_step_overlapped(o, ops); }));
            else
                WW_TRY(replay(o, o->adj_bwd, [&] { return adj_backward_step(o); }));
        }
        launches += (long long)L * o->adj_bwd.nkern;
    }
    c->trans = 0;
    WW_TRY(launch_adj_grad(c, &o->adj, grad));
    c->stats.stages = 8 * c->steps;
    c->stats.launches = c->stream == nullptr ? -1 : launches + 1;
    c->stats.adjoint_bytes = (long long)o->adj.bytes;
    c->stats.device_bytes = (long long)c->dev_bytes;
    c->dtn_ready = false;
    return check_status(c);
}

// ---------------------------------------------------------------- the batch graph
// One RK step of a shot inside the batch graph's WHILE node ends with this
// kernel: it counts the steps and keeps the loop going while steps remain.
__global__ void k_loop_tick(int *count, int steps, cudaGraphConditionalHandle h) {
    const int k = *count + 1;
    *count = k;
    cudaGraphSetConditional(h, k < steps ? 1u : 0u);
}

struct BatchGraph {
    std::vector<unsigned long long> key;      // (id, version) of each context, then the array pointers
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long step_kernels = 0;               // kernels per step of every shot, summed (launch counts)
};

std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch;              // a few recently used batch graphs

void destroy_batch(BatchGraph &b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    b = BatchGraph();
}

void drop_batch_graphs(unsigned long long id) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batch.size();) {
        bool has = false;
        const size_t nctx = g_batch[i].key.empty() ? 0 : (size_t)g_batch[i].key[0];
        for (size_t k = 0; k < nctx && !has; ++k) has = g_batch[i].key[1 + 2 * k] == id;
        if (has) {
            destroy_batch(g_batch[i]);
            g_batch.erase(g_batch.begin() + (long)i);
        } else {
            ++i;
        }
    }
}

// a small graph captured on the context's stream from `body`
template <class F>
int capture_small(Ctx *c, cudaGraph_t *out, F body) {
    *out = nullptr;
    WW_CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    const int st = body();
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != WW_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(WW_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    *out = g;
    return WW_OK;
}

// the branch of shot `o` in the batch graph bg: inputs, initial data, the WHILE
// node of its steps, outputs
int add_batch_branch(cudaGraph_t bg, Owned *o, const double *cvec, double *r, double *J, double *f) {
    Ctx *c = &o->c;
    c->one_col = false;
    WW_TRY(build_prologue_graph(o, 1));
    WW_TRY(build_step_graph(o, 1));
    cudaGraph_t pre = nullptr, post = nullptr;
    WW_TRY(capture_small(c, &pre, [&] {
        WW_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
        WW_CUDA_TRY(cudaMemsetAsync(o->loop_count, 0, sizeof(int), c->stream));
        WW_CUDA_TRY(cudaMemcpyAsync(o->cbuf, cvec, sizeof(double) * (c->n + 1), cudaMemcpyDeviceToDevice, c->stream));
        return WW_OK;
    }));
    int st = capture_small(c, &post, [&] { return launch_outputs(c, r, J, f, 1); });
    cudaGraphNode_t n_pre = nullptr, n_pro = nullptr, n_loop = nullptr, n_post = nullptr, n_step = nullptr,
                    n_tick = nullptr;
    cudaError_t e = cudaSuccess;
    if (st == WW_OK) e = cudaGraphAddChildGraphNode(&n_pre, bg, nullptr, 0, pre);
    if (st == WW_OK && e == cudaSuccess)
        e = cudaGraphAddChildGraphNode(&n_pro, bg, &n_pre, 1, o->prologue[1].graph);
    cudaGraphConditionalHandle h{};
    if (st == WW_OK && e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, bg, 1, cudaGraphCondAssignDefault);
    cudaGraph_t body = nullptr;
    if (st == WW_OK && e == cudaSuccess) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&n_loop, bg, &n_pro, nullptr, 1, &cp);
        if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (st == WW_OK && e == cudaSuccess)
        e = cudaGraphAddChildGraphNode(&n_step, body, nullptr, 0, o->graphs[1][0].graph);
    if (st == WW_OK && e == cudaSuccess) {
        int *cnt = o->loop_count;
        int steps = c->steps;
        void *args[] = {&cnt, &steps, &h};
        cudaKernelNodeParams kp{};
        kp.func = reinterpret_cast<void *>(k_loop_tick);
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(1);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args;
        e = cudaGraphAddKernelNode(&n_tick, body, &n_step, 1, &kp);
    }
    if (st == WW_OK && e == cudaSuccess) e = cudaGraphAddChildGraphNode(&n_post, bg, &n_loop, 1, post);
    if (pre) cudaGraphDestroy(pre);     // the child nodes hold copies
    if (post) cudaGraphDestroy(post);
    if (st != WW_OK) return st;
    if (e != cudaSuccess) return fail(WW_ERR_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    return WW_OK;
}

// ---------------------------------------------------------------- schedules and the autotuner
int check_schedule(const Ctx *c, const ww_schedule &s) {
    if ((s.overlap != 0 && s.overlap != 1) || s.ns_every < 0 || s.ns_every > 2)
        return fail(WW_ERR_ARG, "ww_schedule: overlap must be 0 or 1, ns_every 0, 1 or 2");
    if (s.corr_bn != 32 && s.corr_bn != 64 && s.corr_bn != 128)
        return fail(WW_ERR_ARG, "ww_schedule: corr_bn must be 32, 64 or 128");
    if (s.inv_bn != 64 && s.inv_bn != 128 && s.inv_bn != 256)
        return fail(WW_ERR_ARG, "ww_schedule: inv_bn must be 64, 128 or 256");
    if (s.inv_bn == 256 && c->N % 256 != 0) return fail(WW_ERR_ARG, "ww_schedule: inv_bn 256 needs N % 256 == 0");
    if (s.lu_nb != 32 && s.lu_nb != 64) return fail(WW_ERR_ARG, "ww_schedule: lu_nb must be 32 or 64");
    if (s.inv_ctas != 1 && s.inv_ctas != 2) return fail(WW_ERR_ARG, "ww_schedule: inv_ctas must be 1 or 2");
    if (s.inv_ctas == 2 && s.inv_bn == 256)
        return fail(WW_ERR_ARG, "ww_schedule: inv_ctas 2 needs inv_bn 64 or 128");
    if (s.prio != 0 && s.prio != 1) return fail(WW_ERR_ARG, "ww_schedule: prio must be 0 or 1");
    return WW_OK;
}

int apply_schedule(Owned *o, const ww_schedule &s) {
    Ctx *c = &o->c;
    WW_TRY(check_schedule(c, s));
    if (std::memcmp(&c->sch, &s, sizeof(s)) == 0) return WW_OK;
    WW_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (o->side_stream) WW_CUDA_TRY(cudaStreamSynchronize(o->side_stream));
    drop_graphs(o);
    c->sch = s;
    // the LU block (the inverted diagonal blocks' buffer is sized for LU_NB, the largest)
    c->nb = c->N < s.lu_nb ? c->N : s.lu_nb;
    return WW_OK;
}

std::string tune_key(const Ctx *c) {
    std::ostringstream k;
    k << c->N << " " << c->nc << " " << (c->precision == WW_MIXED ? "mixed" : "fp64");
    return k.str();
}

// the cached schedule of this (N, n+1, precision), if the file has one; lines
// read "v2 N n+1 form overlap ns_every corr_bn inv_bn lu_nb inv_ctas prio ms"
// (lines of another layout are passed over)
bool cache_lookup(const char *path, const std::string &key, ww_schedule *out) {
    if (!path) return false;
    std::ifstream in(path);
    std::string line;
    bool found = false;
    while (std::getline(in, line)) {
        std::istringstream ls(line);
        int N = 0, nc = 0;
        std::string tag, form;
        ww_schedule s{};
        if (!(ls >> tag) || tag != "v2") continue;
        if (!(ls >> N >> nc >> form >> s.overlap >> s.ns_every >> s.corr_bn >> s.inv_bn >> s.lu_nb >> s.inv_ctas >>
              s.prio))
            continue;
        std::ostringstream k;
        k << N << " " << nc << " " << form;
        if (k.str() == key) {
            *out = s;
            found = true;   // the last line for a key wins
        }
    }
    return found;
}

int cache_store(const char *path, const std::string &key, const ww_schedule &s, double ms) {
    if (!path) return WW_OK;
    std::ofstream out(path, std::ios::app);
    if (!out) return fail(WW_ERR_ARG, std::string("ww_autotune: cannot append to ") + path);
    out << "v2 " << key << " " << s.overlap << " " << s.ns_every << " " << s.corr_bn << " " << s.inv_bn << " "
        << s.lu_nb << " " << s.inv_ctas << " " << s.prio << " " << ms << "\n";
    return WW_OK;
}

// ms per RK step of the Jacobian program under schedule s: initial data, one
// untimed step (captures the program), probe steps timed with events
int probe_schedule(Owned *o, const ww_schedule &s, int probe_steps, double *ms) {
    Ctx *c = &o->c;
    WW_TRY(apply_schedule(o, s));
    c->one_col = false;
    WW_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    WW_TRY(run_prologue(o, 1));
    WW_TRY(build_step_graph(o, 1));
    const cudaGraphExec_t ex = o->graphs[1][0].exec;
    WW_CUDA_TRY(cudaGraphLaunch(ex, c->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    WW_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
    for (int k = 0; k < probe_steps && e == cudaSuccess; ++k) e = cudaGraphLaunch(ex, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return fail(WW_ERR_CUDA, std::string("ww_autotune probe: ") + cudaGetErrorString(e));
    const int stt = check_status(c);   // a schedule that fails to converge is not a candidate
    *ms = stt == WW_OK ? (double)t / probe_steps : INFINITY;
    return WW_OK;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

}  // namespace

int phase_mark(Ctx *c, int phase, int b) { return mark(c, c->cur_stage, phase, b); }

Ctx *ctx_of(ww_ctx *h) { return &owner(h)->c; }

int read_status(Ctx *c) { return check_status(c); }

}  // namespace ww

using namespace ww;

extern "C" {

const char *ww_last_error(void) { return g_err.c_str(); }

int ww_create(ww_ctx **out, const ww_problem *p) {
    if (!out || !p) return fail(WW_ERR_ARG, "ww_create: NULL argument");
    *out = nullptr;
    if (!is_pow2(p->N) || p->N < 16 || p->N > 4096)
        return fail(WW_ERR_ARG, "ww_create: N must be a power of two in [16, 4096]");
    if (p->n < 0 || p->n > 4096) return fail(WW_ERR_ARG, "ww_create: n must be in [0, 4096]");
    if (p->steps < 1) return fail(WW_ERR_ARG, "ww_create: steps must be >= 1");
    if (!std::isfinite(p->g) || !std::isfinite(p->tau) || p->tau < 0.0)
        return fail(WW_ERR_ARG, "ww_create: g and tau must be finite, tau >= 0");
    if (!(p->h > 0.0)) return fail(WW_ERR_ARG, "ww_create: h must be > 0 (INFINITY for deep water)");
    if (p->precision != WW_FP64 && p->precision != WW_MIXED)
        return fail(WW_ERR_ARG, "ww_create: precision must be WW_FP64 or WW_MIXED");
    if (p->precision == WW_MIXED && p->N < 64)
        return fail(WW_ERR_ARG, "ww_create: WW_MIXED needs N >= 64 (64-wide tensor-core K tiles)");

    Owned *o = new Owned();
    Ctx *c = &o->c;
    std::memset(c, 0, sizeof(Ctx));
    c->N = p->N;
    c->logN = 0;
    while ((1 << c->logN) < c->N) ++c->logN;
    c->n = p->n;
    c->nc = p->n + 1;
    c->NC = c->nc + 1;
    c->g = p->g;
    c->tau = p->tau;
    c->h = p->h;
    c->deep = std::isinf(p->h);
    c->steps = p->steps;
    c->precision = p->precision;
    c->refine_tol = p->refine_tol > 0.0 ? p->refine_tol : 1e-13;
    c->max_refine = p->max_refine > 0 ? p->max_refine : 4;
    c->sch = ww_schedule{1, 2, 64, 128, LU_NB, 2, 1};
    c->nb = c->N < LU_NB ? c->N : LU_NB;
    {
        static std::atomic<unsigned long long> next_id{1};
        o->id = next_id++;
    }
    {
        cudaError_t e0 = cudaStreamCreateWithFlags(&o->own_stream, cudaStreamNonBlocking);
        if (e0 != cudaSuccess) {
            delete o;
            return fail(WW_ERR_CUDA, std::string("ww_create stream: ") + cudaGetErrorString(e0));
        }
    }
    c->stream = o->own_stream;
    c->owner = o;
    {
        // the base chain is latency bound: its blocks go first when SMs free up
        int lo = 0, hi = 0;
        cudaError_t e0 = cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (e0 == cudaSuccess) e0 = cudaStreamCreateWithPriority(&o->side_stream, cudaStreamNonBlocking, hi);
        if (e0 == cudaSuccess) e0 = cudaEventCreateWithFlags(&o->ev_fork, cudaEventDisableTiming);
        if (e0 == cudaSuccess) e0 = cudaEventCreateWithFlags(&o->ev_join, cudaEventDisableTiming);
        for (int k = 0; k < 4 && e0 == cudaSuccess; ++k) {
            e0 = cudaEventCreateWithFlags(&o->ev_base[k], cudaEventDisableTiming);
            if (e0 == cudaSuccess) e0 = cudaEventCreateWithFlags(&o->ev_cols[k], cudaEventDisableTiming);
        }
        if (e0 != cudaSuccess) {
            ww_destroy(reinterpret_cast<ww_ctx *>(o));
            return fail(WW_ERR_CUDA, std::string("ww_create streams/events: ") + cudaGetErrorString(e0));
        }
    }

    const size_t N = c->N, NC = c->NC, nb = c->nb;
    const size_t nblk = (N + nb - 1) / nb;
    int st = WW_OK;
#define ALLOC(ptr, cnt)                                     \
    if (st == WW_OK) st = dalloc_n(o, &(ptr), (size_t)(cnt))
    ALLOC(c->tw, N / 2);
    if (p->precision == WW_MIXED) ALLOC(c->twd, N / 2);
    ALLOC(c->cs, 3 * N);
    ALLOC(c->eta, N);
    ALLOC(c->eta_x, N);
    ALLOC(c->eta_xx, N);
    ALLOC(c->phi_s, N);
    ALLOC(c->E, N);
    ALLOC(c->Einv, N);
    for (int q = 0; q < 2; ++q) {
        ALLOC(c->ux_p[q], N);
        ALLOC(c->vy_p[q], N);
        ALLOC(c->w3_p[q], N);
        ALLOC(c->Fbase_p[q], 2 * N);
        if (p->precision == WW_MIXED) {
            ALLOC(c->uxd_p[q], N);
            ALLOC(c->vyd_p[q], N);
            ALLOC(c->w3d_p[q], N);
        }
    }
    ALLOC(c->filt_d, N);
    if (p->precision == WW_MIXED) ALLOC(c->filt_df, N);
    ALLOC(c->curv, N);
    ALLOC(c->A, N * N);
    ALLOC(c->G, N * N);
    ALLOC(c->Dinv, nblk * 2 * nb * nb);
    ALLOC(c->Y, NC * 2 * N);
    ALLOC(c->Ys, NC * 2 * N);
    ALLOC(c->Kacc, NC * 2 * N);
    ALLOC(c->M, N * NC);
    ALLOC(c->Gam, N * NC);
    ALLOC(c->Gout, N * NC);
    ALLOC(c->basis, 2 * N * (size_t)(p->n > 0 ? p->n : 1));
    ALLOC(c->status, 1);
    ALLOC(c->small, 64);
    ALLOC(o->cbuf, c->n + 1);
    ALLOC(o->rbuf, N);
    ALLOC(o->Jbuf, N * c->nc);
    ALLOC(o->fbuf, 1);
    ALLOC(o->loop_count, 1);
#undef ALLOC
    if (st != WW_OK) {
        ww_destroy(reinterpret_cast<ww_ctx *>(o));
        return st;
    }
    select_parity(c, 0);
    std::vector<double> tw(N), cs(3 * N);
    fill_tables(c->N, tw.data(), cs.data());
    const double two_pi = 6.283185307179586476925286766559;
    std::vector<double> basis(2 * N * (size_t)(p->n > 0 ? p->n : 1), 0.0);
    for (int k = 0; k < p->n; ++k)
        for (size_t r = 0; r < 2 * N; ++r)
            basis[(size_t)k * 2 * N + r] =
                p->basis ? p->basis[(size_t)k * 2 * N + r]
                         : (r < N ? std::cos((double)(k + 1) * two_pi * (double)r / (double)N) : 0.0);
    cudaError_t e = cudaMemcpy(c->tw, tw.data(), sizeof(double) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->cs, cs.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->basis, basis.data(), sizeof(double) * basis.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(int));
    if (e == cudaSuccess && c->twd) {
        // double-float twiddles: hi = float(w), lo = float(w - hi)
        std::vector<float> twd(2 * N);
        for (size_t k = 0; k < N; ++k) {
            const float hi = (float)tw[k];
            twd[2 * k] = hi;
            twd[2 * k + 1] = (float)(tw[k] - (double)hi);
        }
        e = cudaMemcpy(c->twd, twd.data(), sizeof(float) * 2 * N, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        ww_destroy(reinterpret_cast<ww_ctx *>(o));
        return fail(WW_ERR_CUDA, std::string("ww_create upload: ") + cudaGetErrorString(e));
    }
    st = prepare_spectral(c);
    if (st == WW_OK) st = launch_fill_filter(c);
    if (st == WW_OK && cudaStreamSynchronize(c->stream) != cudaSuccess) st = fail(WW_ERR_CUDA, "ww_create: filter tables");
    if (st == WW_OK) st = prepare_dense();
    if (st != WW_OK) {
        ww_destroy(reinterpret_cast<ww_ctx *>(o));
        return st;
    }
    if (c->precision == WW_MIXED) {
        st = mixed_create(c);
        if (st != WW_OK) {
            ww_destroy(reinterpret_cast<ww_ctx *>(o));
            return st;
        }
    }
    *out = reinterpret_cast<ww_ctx *>(o);
    g_err.clear();
    return WW_OK;
}

void ww_destroy(ww_ctx *ctx) {
    if (!ctx) return;
    Owned *o = owner(ctx);
    drop_batch_graphs(o->id);
    for (int w = 0; w < 2; ++w) {
        for (int t = 0; t < 2; ++t) {
            if (o->graphs[w][t].exec) cudaGraphExecDestroy(o->graphs[w][t].exec);
            if (o->graphs[w][t].graph) cudaGraphDestroy(o->graphs[w][t].graph);
        }
        if (o->prologue[w].exec) cudaGraphExecDestroy(o->prologue[w].exec);
        if (o->prologue[w].graph) cudaGraphDestroy(o->prologue[w].graph);
    }
    for (StepGraph *sg : {&o->adj_fwd, &o->adj_mid, &o->adj_bwd, &o->adj_restart, &o->adj_reentry}) {
        if (sg->exec) cudaGraphExecDestroy(sg->exec);
        if (sg->graph) cudaGraphDestroy(sg->graph);
    }
    for (cudaEvent_t ev : o->placeholder)
        if (ev) cudaEventDestroy(ev);
    for (cudaEvent_t ev : o->pool) cudaEventDestroy(ev);
    if (o->c.mx) mixed_destroy(&o->c);
    if (o->c.seg) segment_destroy(&o->c);
    if (o->c.stream) cudaStreamSynchronize(o->c.stream);
    if (o->side_stream) cudaStreamSynchronize(o->side_stream);
    for (void *p : o->allocs) cudaFree(p);
    if (o->own_stream) cudaStreamDestroy(o->own_stream);
    if (o->side_stream) cudaStreamDestroy(o->side_stream);
    cudaEvent_t evs[] = {o->ev_fork, o->ev_join, o->ev_base[0], o->ev_base[1], o->ev_base[2], o->ev_base[3],
                         o->ev_cols[0], o->ev_cols[1], o->ev_cols[2], o->ev_cols[3]};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    delete o;
}

int ww_set_stream(ww_ctx *ctx, void *stream) {
    if (!ctx) return fail(WW_ERR_ARG, "ww_set_stream: NULL context");
    Owned *o = owner(ctx);
    // graphs are replayed on whatever stream is current, so nothing is rebuilt;
    // the legacy default stream (NULL) selects direct launches instead of graphs
    o->c.stream = (cudaStream_t)stream;
    return WW_OK;
}

int ww_set_timing(ww_ctx *ctx, int enable) {
    if (!ctx) return fail(WW_ERR_ARG, "ww_set_timing: NULL context");
    owner(ctx)->timing = enable != 0;
    return WW_OK;
}

int ww_get_timing(const ww_ctx *ctx, double *ms, int *launches) {
    if (!ctx || !ms || !launches) return fail(WW_ERR_ARG, "ww_get_timing: NULL argument");
    const Owned *o = reinterpret_cast<const Owned *>(ctx);
    for (int p = 0; p < NPH; ++p) {
        ms[p] = o->ph_ms[p];
        launches[p] = o->ph_count[p];
    }
    return WW_OK;
}

int ww_set_verify(ww_ctx *ctx, int every) {
    if (!ctx) return fail(WW_ERR_ARG, "ww_set_verify: NULL context");
    if (every < 0) return fail(WW_ERR_ARG, "ww_set_verify: every must be >= 0");
    Owned *o = owner(ctx);
    if (o->c.precision != WW_MIXED && every > 0)
        return fail(WW_ERR_ARG, "ww_set_verify: only WW_MIXED has a refinement residual to measure");
    if (o->c.verify_every == every) return WW_OK;
    WW_CUDA_TRY(cudaStreamSynchronize(o->c.stream));
    if (o->side_stream) WW_CUDA_TRY(cudaStreamSynchronize(o->side_stream));
    // the step programs captured so far were built without (or with) the measurement
    drop_graphs(o);
    o->c.verify_every = every;
    return WW_OK;
}

int ww_set_checkpoint(ww_ctx *ctx, int every) {
    if (!ctx) return fail(WW_ERR_ARG, "ww_set_checkpoint: NULL context");
    if (every < 0) return fail(WW_ERR_ARG, "ww_set_checkpoint: every must be >= 0");
    Owned *o = owner(ctx);
    WW_CUDA_TRY(cudaStreamSynchronize(o->c.stream));
    if (o->side_stream) WW_CUDA_TRY(cudaStreamSynchronize(o->side_stream));
    o->c.ckpt_every = every;   // the adjoint workspace is resized by the next objective_and_grad
    return WW_OK;
}

int ww_get_stats(const ww_ctx *ctx, ww_stats *out) {
    if (!ctx || !out) return fail(WW_ERR_ARG, "ww_get_stats: NULL argument");
    *out = reinterpret_cast<const Owned *>(ctx)->c.stats;
    return WW_OK;
}

int dtn_setup(ww_ctx *ctx, const double *eta) {
    if (!ctx || !eta) return fail(WW_ERR_ARG, "dtn_setup: NULL argument");
    Ctx *c = &owner(ctx)->c;
    c->dtn_ready = false;
    c->one_col = false;   // dtn_apply may take many columns
    select_parity(c, 0);
    WW_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    WW_TRY(launch_base_geometry(c, eta, nullptr, 0));
    WW_TRY(launch_assemble(c));
    WW_TRY(factor(c, 1));
    WW_TRY(check_status(c));
    c->dtn_ready = true;
    return WW_OK;
}

int dtn_apply(ww_ctx *ctx, const double *phi, int nrhs, double *Gphi) {
    if (!ctx || !phi || !Gphi) return fail(WW_ERR_ARG, "dtn_apply: NULL argument");
    Ctx *c = &owner(ctx)->c;
    if (!c->dtn_ready) return fail(WW_ERR_ARG, "dtn_apply: call dtn_setup first");
    if (nrhs < 1 || nrhs > c->NC) return fail(WW_ERR_ARG, "dtn_apply: nrhs must be in [1, n + 2]");
    WW_CUDA_TRY(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    WW_TRY(launch_copy_cols(c, phi, nrhs, c->M));
    WW_TRY(solve(c, c->M, nrhs));
    WW_TRY(launch_gamma(c, 0, nrhs));
    WW_TRY(apply_G(c, 0, nrhs));
    WW_TRY(launch_copy_cols(c, c->Gout, nrhs, Gphi));
    return check_status(c);
}

int shoot(ww_ctx *ctx, const double *cvec, double *r, double *f) {
    if (!ctx || !cvec || !r || !f) return fail(WW_ERR_ARG, "shoot: NULL argument");
    return run_shot(owner(ctx), cvec, false, r, nullptr, f, 0);
}

int shoot_jacobian(ww_ctx *ctx, const double *cvec, double *r, double *J, double *f) {
    if (!ctx || !cvec || !r || !J || !f) return fail(WW_ERR_ARG, "shoot_jacobian: NULL argument");
    return run_shot(owner(ctx), cvec, false, r, J, f, 1);
}

int shoot_jacobian_host(ww_ctx *ctx, const double *cvec, double *r, double *J, double *f) {
    if (!ctx || !cvec || !r || !J || !f) return fail(WW_ERR_ARG, "shoot_jacobian_host: NULL argument");
    Owned *o = owner(ctx);
    Ctx *c = &o->c;
    WW_TRY(run_shot(o, cvec, true, o->rbuf, o->Jbuf, o->fbuf, 1));
    WW_CUDA_TRY(cudaMemcpyAsync(r, o->rbuf, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaMemcpyAsync(J, o->Jbuf, sizeof(double) * c->N * c->nc, cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaMemcpyAsync(f, o->fbuf, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    WW_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return WW_OK;
}

int shoot_jacobian_batch(ww_ctx *const *ctx, int nshots, const double *const *cvec, double *const *r,
                         double *const *J, double *const *f) {
    if (nshots < 0 || (nshots > 0 && (!ctx || !cvec || !r || !J || !f)))
        return fail(WW_ERR_ARG, "shoot_jacobian_batch: NULL argument");
    if (nshots == 0) return WW_OK;
    for (int i = 0; i < nshots; ++i) {
        if (!ctx[i] || !cvec[i] || !r[i] || !J[i] || !f[i])
            return fail(WW_ERR_ARG, "shoot_jacobian_batch: NULL entry for shot " + std::to_string(i));
        if (owner(ctx[i])->c.stream == nullptr)
            return fail(WW_ERR_ARG, "shoot_jacobian_batch: shot " + std::to_string(i) +
                                        " runs on the legacy default stream (the shots need streams of their own)");
        for (int k = 0; k < i; ++k)
            if (ctx[k] == ctx[i] || owner(ctx[k])->c.stream == owner(ctx[i])->c.stream)
                return fail(WW_ERR_ARG, "shoot_jacobian_batch: shots " + std::to_string(k) + " and " +
                                            std::to_string(i) + " share a context or a stream");
    }
    // the batch replays each shot's untimed step program; timing flags come back on return
    struct TimingGuard {
        std::vector<std::pair<Owned *, bool>> saved;
        ~TimingGuard() {
            for (auto &p : saved) p.first->timing = p.second;
        }
    } guard;
    std::vector<unsigned long long> key{(unsigned long long)nshots};
    for (int i = 0; i < nshots; ++i) {
        Owned *o = owner(ctx[i]);
        guard.saved.emplace_back(o, o->timing);
        o->timing = false;
        key.push_back(o->id);
        key.push_back(o->version);
    }
    for (int i = 0; i < nshots; ++i)
        for (const void *p : {(const void *)cvec[i], (const void *)r[i], (const void *)J[i], (const void *)f[i]})
            key.push_back((unsigned long long)(uintptr_t)p);
    Owned *o0 = owner(ctx[0]);
    cudaStream_t s0 = o0->c.stream;
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_batch_mu);
        for (size_t i = 0; i < g_batch.size(); ++i)
            if (g_batch[i].key == key) {
                std::rotate(g_batch.begin(), g_batch.begin() + (long)i, g_batch.begin() + (long)i + 1);
                exec = g_batch[0].exec;
                break;
            }
    }
    if (!exec) {
        BatchGraph b;
        b.key = key;
        WW_CUDA_TRY(cudaGraphCreate(&b.graph, 0));
        int st = WW_OK;
        for (int i = 0; i < nshots && st == WW_OK; ++i) {
            Owned *o = owner(ctx[i]);
            st = add_batch_branch(b.graph, o, cvec[i], r[i], J[i], f[i]);
            if (st != WW_OK) st = fail(st, "shot " + std::to_string(i) + ": " + ww_last_error());
            else b.step_kernels += o->graphs[1][0].nkern;
        }
        if (st == WW_OK) {
            const cudaError_t e = cudaGraphInstantiate(&b.exec, b.graph, 0);
            if (e != cudaSuccess) st = fail(WW_ERR_CUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(e));
        }
        if (st != WW_OK) {
            destroy_batch(b);
            return st;
        }
        exec = b.exec;
        std::lock_guard<std::mutex> lk(g_batch_mu);
        g_batch.insert(g_batch.begin(), b);
        while (g_batch.size() > 4) {
            destroy_batch(g_batch.back());
            g_batch.pop_back();
        }
    }
    // one launch on the first shot's stream, ordered after the other shots' streams
    for (int i = 1; i < nshots; ++i) {
        Owned *o = owner(ctx[i]);
        WW_CUDA_TRY(cudaEventRecord(o->ev_join, o->c.stream));
        WW_CUDA_TRY(cudaStreamWaitEvent(s0, o->ev_join, 0));
    }
    WW_CUDA_TRY(cudaGraphLaunch(exec, s0));
    WW_CUDA_TRY(cudaEventRecord(o0->ev_join, s0));
    for (int i = 1; i < nshots; ++i) WW_CUDA_TRY(cudaStreamWaitEvent(owner(ctx[i])->c.stream, o0->ev_join, 0));
    for (int i = 0; i < nshots; ++i) {
        Owned *o = owner(ctx[i]);
        Ctx *c = &o->c;
        c->stats.stages = 4 * c->steps;
        // prologue, steps x (step program + the loop counter), outputs
        c->stats.launches = (long long)o->prologue[1].nkern + (long long)c->steps * (o->graphs[1][0].nkern + 1) + 2;
        c->stats.device_bytes = (long long)c->dev_bytes;
        c->dtn_ready = false;
    }
    for (int i = 0; i < nshots; ++i) {
        const int st = check_status(&owner(ctx[i])->c);
        if (st != WW_OK) return fail(st, "shot " + std::to_string(i) + ": " + ww_last_error());
    }
    return WW_OK;
}

int ww_set_schedule(ww_ctx *ctx, const ww_schedule *s) {
    if (!ctx || !s) return fail(WW_ERR_ARG, "ww_set_schedule: NULL argument");
    return apply_schedule(owner(ctx), *s);
}

int ww_get_schedule(const ww_ctx *ctx, ww_schedule *s) {
    if (!ctx || !s) return fail(WW_ERR_ARG, "ww_get_schedule: NULL argument");
    *s = reinterpret_cast<const Owned *>(ctx)->c.sch;
    return WW_OK;
}

int ww_autotune(ww_ctx *ctx, const double *cvec, int probe_steps, const char *cache_path, double *ms_per_step) {
    if (!ctx || !cvec) return fail(WW_ERR_ARG, "ww_autotune: NULL argument");
    if (probe_steps < 1) return fail(WW_ERR_ARG, "ww_autotune: probe_steps must be >= 1");
    Owned *o = owner(ctx);
    Ctx *c = &o->c;
    if (c->stream == nullptr) return fail(WW_ERR_ARG, "ww_autotune: the legacy default stream runs no step graphs");
    if (ms_per_step) *ms_per_step = 0.0;
    const std::string key = tune_key(c);
    ww_schedule best = c->sch;
    if (cache_lookup(cache_path, key, &best)) return apply_schedule(o, best);
    const bool timing = o->timing;
    o->timing = false;
    struct Restore {
        Owned *o;
        bool t;
        ~Restore() { o->timing = t; }
    } restore{o, timing};
    WW_CUDA_TRY(cudaMemcpyAsync(o->cbuf, cvec, sizeof(double) * (c->n + 1), cudaMemcpyDeviceToDevice, c->stream));
    double best_ms = INFINITY;
    auto consider = [&](ww_schedule s) -> int {
        double ms = INFINITY;
        WW_TRY(probe_schedule(o, s, probe_steps, &ms));
        if (ms < best_ms) {
            best_ms = ms;
            best = s;
        }
        return WW_OK;
    };
    // coordinate by coordinate from the default schedule
    ww_schedule base = ww_schedule{1, 2, 64, 128, LU_NB, 2, 1};
    if (c->precision == WW_MIXED) {
        // stage program: in line, overlapped with every-stage, alternate, or alternate
        // until odd stages need a third correction
        for (int v : {0, 1, 2, 3}) {
            ww_schedule s = base;
            s.overlap = v > 0;
            s.ns_every = v == 1 ? 1 : (v == 3 ? 2 : 0);
            WW_TRY(consider(s));
        }
        base = best;
        for (int bn : {32, 128}) {
            ww_schedule s = base;
            s.corr_bn = bn;
            WW_TRY(consider(s));
        }
        base = best;
        for (int bn : {64, 256}) {   // (256-wide tiles take one CTA per SM)
            if (bn == 256 && c->N % 256 != 0) continue;
            ww_schedule s = base;
            s.inv_bn = bn;
            if (bn == 256) s.inv_ctas = 1;
            WW_TRY(consider(s));
        }
        if (best.inv_bn != 256) {
            ww_schedule s = best;
            s.inv_ctas = 3 - best.inv_ctas;
            WW_TRY(consider(s));
        }
        if (best.overlap) {
            ww_schedule s = best;
            s.prio = 1 - best.prio;
            WW_TRY(consider(s));
        }
    } else {
        for (int nb : {64, 32}) {
            ww_schedule s = base;
            s.lu_nb = nb;
            WW_TRY(consider(s));
        }
    }
    if (!std::isfinite(best_ms)) return fail(WW_ERR_NO_CONVERGENCE, "ww_autotune: no candidate schedule converged");
    WW_TRY(apply_schedule(o, best));
    if (ms_per_step) *ms_per_step = best_ms;
    return cache_store(cache_path, key, best, best_ms);
}

int objective_and_grad(ww_ctx *ctx, const double *cvec, double *f, double *grad) {
    if (!ctx || !cvec || !f || !grad) return fail(WW_ERR_ARG, "objective_and_grad: NULL argument");
    Owned *o = owner(ctx);
    WW_TRY(run_adjoint(o, cvec, false, f, grad));
    WW_CUDA_TRY(cudaStreamSynchronize(o->c.stream));
    return WW_OK;
}

}  // extern "C"
