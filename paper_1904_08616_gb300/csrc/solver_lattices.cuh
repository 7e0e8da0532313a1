// Several lattices of different sizes solved together (Algorithm 1 for each).  The paper
// solves one system at a time; this is the library's batching of uneven problems.
//
// Each lattice keeps its own solver (state record, fields, kernels with the grids a solve of
// that lattice alone would use).  By default the whole batch is one CUDA graph
// (LatticeSolveGraph): rounds of cycles with each lattice's outer steps (restart, reliable
// update) and every decision on the device, and in the inner loop each lattice's K1, K2, K3
// as a parallel branch of the graph, so that the small lattices' kernels run beside the large
// one's instead of after them.  Host-driven forms remain for LQ_CG_LATTICE_OWN_CYCLES (a
// conditional graph over the inner iterations that returns when one lattice's cycle ends),
// for LQ_CG_NO_GRAPH and for drivers without nested conditional nodes: they issue the
// lattices' inner kernels one lattice after the other, the host reads the state records
// between launches and runs the outer steps of the lattices whose cycle ended, on the same
// stream.  Every form gives each lattice the sums of its own solve, bit for bit.  Lattices
// whose inner loop has stopped leave their kernels idle.
//
// The inner block size (threads per block of K1/K2) is a template parameter; the tuner
// times K1 over the actual lattices for each candidate and caches the winner by a JSON key
// (GPU, mode, lattice shapes and right-hand-side counts), in memory and, when the
// environment variable LQ_TUNE_CACHE names a file, on disk.
#pragma once

#include <memory>
#include <string>

#include "solver_impl.cuh"

namespace lq {

namespace solver_detail {

constexpr int kMaxLat = 8;

// One inner iteration of every lattice of a batch: each lattice's K1, K2, K3 are its own
// launches, with the grids a solve of that lattice alone would use (so each lattice's sums
// are those of its own solve, bit for bit).  iteration() issues them one lattice after the
// other on one stream (host-driven cycles); iteration_of(l, s) issues lattice l's on s, the
// branch of a graph in which the lattices' kernels run side by side.
template <class S> struct InnerLaunches {
    const S* sv = nullptr;
    int n = 0;
    void build(const S* sv_, int n_) {
        sv = sv_;
        n = n_;
    }
    cudaError_t k1_only(cudaStream_t s) const {
        cudaError_t e = cudaSuccess;
        for (int l = 0; l < n && e == cudaSuccess; ++l) e = sv[l].launch_k1(s);
        return e;
    }
    cudaError_t iteration(cudaStream_t s) const {
        cudaError_t e = cudaSuccess;
        for (int l = 0; l < n && e == cudaSuccess; ++l) e = sv[l].launch_iteration(s);
        return e;
    }
    cudaError_t iteration_of(int l, cudaStream_t s) const { return sv[l].launch_iteration(s); }
};

// One lattice of a multi-lattice solve as the drivers see it.
struct LatticeJob {
    Geom g;
    double m_q;
    int nb;
    const void* U;
    const void* eta;
    void* x;
    WsLayout w;
    size_t off;   // byte offset of its workspace
};

// chunk x {K1, K2, K3} captured on a private stream, replayed on the caller's stream
struct ChunkGraph {
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ChunkGraph() = default;
    ChunkGraph(const ChunkGraph&) = delete;
    ChunkGraph& operator=(const ChunkGraph&) = delete;
    ~ChunkGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
    }
    template <class IL>
    cudaError_t capture(const IL& il, int chunk) {
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
        cudaError_t le = cudaSuccess;
        for (int j = 0; j < chunk && le == cudaSuccess; ++j) le = il.iteration(cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (le != cudaSuccess) return le;
        if (e != cudaSuccess) return e;
        return cudaGraphInstantiate(&exec, graph, 0);
    }
};

// The batch's inner loop on the device: a prologue kernel records how many lattices are idle
// (all_stop set) and the trip bound, then a conditional WHILE node repeats one iteration of
// every lattice and a one-thread condition kernel until some running lattice stops (its
// cycle then ends on the host), every lattice is idle, or the bound is reached.  The counters
// live in the first lattice's state record.
struct LatLoopArgs {
    SolverState* st[kMaxLat];
    int n;
    int together;   // run until every lattice's inner loop has stopped (else until one has)
};

static __global__ void lattice_loop_base(LatLoopArgs a) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int idle = 0, cap = 0;
        for (int l = 0; l < a.n; ++l) {
            if (a.st[l]->all_stop) ++idle;
            else cap = max(cap, a.st[l]->k_max);
        }
        a.st[0]->loop_base = idle;
        a.st[0]->loop_trips = 0;
        a.st[0]->loop_cap = cap + 2;
    }
}

static __global__ void lattice_loop_cond(cudaGraphConditionalHandle h, LatLoopArgs a) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int idle = 0;
        for (int l = 0; l < a.n; ++l) idle += a.st[l]->all_stop ? 1 : 0;
        SolverState* s0 = a.st[0];
        const int t = ++s0->loop_trips;
        const bool more = a.together ? idle < a.n : (idle == s0->loop_base && idle < a.n);
        cudaGraphSetConditional(h, (more && t < s0->loop_cap) ? 1u : 0u);
    }
}

struct LoopGraph {
    cudaStream_t cs = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    LoopGraph() = default;
    LoopGraph(const LoopGraph&) = delete;
    LoopGraph& operator=(const LoopGraph&) = delete;
    ~LoopGraph() { reset(); }
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cs) cudaStreamDestroy(cs);
        exec = nullptr;
        graph = nullptr;
        cs = nullptr;
    }
    template <class IL>
    cudaError_t build(const IL& il, const LatLoopArgs& a) {
        cudaError_t e;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess) return e;
        // prologue node
        cudaKernelNodeParams kp = {};
        LatLoopArgs args = a;
        void* kargs[] = {&args};
        kp.func = (void*)lattice_loop_base;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.kernelParams = kargs;
        cudaGraphNode_t base;
        if ((e = cudaGraphAddKernelNode(&base, graph, nullptr, 0, &kp)) != cudaSuccess) return e;
        // WHILE node after it
        cudaGraphConditionalHandle h;
        if ((e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        if ((e = cudaGraphAddNode(&node, graph, &base, nullptr, 1, &p)) != cudaSuccess) return e;
        cudaGraph_t bodyg = p.conditional.phGraph_out[0];
        if ((e = cudaStreamBeginCaptureToGraph(cs, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            return e;
        cudaError_t le = il.iteration(cs);
        if (le == cudaSuccess) {
            lattice_loop_cond<<<1, 32, 0, cs>>>(h, a);
            le = cudaGetLastError();
        }
        e = cudaStreamEndCapture(cs, &bodyg);
        if (le != cudaSuccess) return le;
        if (e != cudaSuccess) return e;
        return cudaGraphInstantiate(&exec, graph, 0);
    }
};

// A lattice batch's whole solve as one CUDA graph (reliable updates taken together, every
// decision on the device):
//   lat_first; WHILE (some lattice needs a cycle) { arm; restart of every lattice;
//   lattice_loop_base; WHILE (some lattice's inner loop runs) { one iteration of every
//   lattice; lattice_loop_cond }; for each lattice { lat_mid; IF (its solution moved)
//   { its update and outer residual; lat_end } }; lat_decide }
// The lattices' kernels are parallel branches of the graph, so a small lattice's kernels run
// beside a large one's.  A lattice with nothing left to do takes part with idle kernels and
// no-op cycle kernels.
struct LatCtlArgs {
    SolverState* st[kMaxLat];
    int n;
};
static __global__ void lat_first_kernel(LatCtlArgs a, cudaGraphConditionalHandle outer) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        bool any = false;
        for (int l = 0; l < a.n; ++l) {
            CycleCtl& c = a.st[l]->ctl;
            const bool w = ctl_plan(c);
            ctl_params(c);
            c.want = w;
            c.launches += 1;
            any |= w;
        }
        cudaGraphSetConditional(outer, any ? 1u : 0u);
    }
}
static __global__ void lat_mid_kernel(SolverState* st, cudaGraphConditionalHandle run) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        CycleCtl& c = st->ctl;
        ctl_mid(c, *st);
        int moved = 0;
        for (int j = 0; j < kMaxRhs; ++j) moved |= c.xact[j];
        if (!moved) c.want = 0;
        cudaGraphSetConditional(run, moved ? 1u : 0u);
    }
}
static __global__ void lat_end_kernel(SolverState* st) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        CycleCtl& c = st->ctl;
        ctl_collect(c, *st);
        c.want = ctl_plan(c);
        ctl_params(c);
    }
}
// launches per round charged to every lattice: arm, base, decide, its two restart kernels and
// lat_mid, four per inner trip (three shared iteration kernels and the loop test), and its
// update, two residual kernels and lat_end when its solution moved
static __global__ void lat_decide_kernel(LatCtlArgs a, cudaGraphConditionalHandle outer) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        bool any = false;
        const int trips = a.st[0]->loop_trips;
        for (int l = 0; l < a.n; ++l) {
            CycleCtl& c = a.st[l]->ctl;
            int moved = 0;
            for (int j = 0; j < kMaxRhs; ++j) moved |= c.xact[j];
            c.launches += 6 + 4 * trips + (moved ? 4 : 0);
            any |= c.want != 0;
        }
        cudaGraphSetConditional(outer, any ? 1u : 0u);
    }
}

struct LatticeSolveGraph {
    cudaStream_t cs = nullptr;
    cudaStream_t ls[kMaxLat] = {};   // one capture branch per lattice
    cudaEvent_t ev[kMaxLat + 1] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int n = 0;
    LatticeSolveGraph() = default;
    LatticeSolveGraph(const LatticeSolveGraph&) = delete;
    LatticeSolveGraph& operator=(const LatticeSolveGraph&) = delete;
    ~LatticeSolveGraph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (int l = 0; l < kMaxLat; ++l)
            if (ls[l]) cudaStreamDestroy(ls[l]);
        for (int l = 0; l <= kMaxLat; ++l)
            if (ev[l]) cudaEventDestroy(ev[l]);
        if (cs) cudaStreamDestroy(cs);
    }
    // while cs is capturing: f(l, ls[l]) for every lattice as parallel branches, joined on cs
    template <class F>
    cudaError_t branches(F f) {
        cudaError_t e;
        if ((e = cudaEventRecord(ev[kMaxLat], cs)) != cudaSuccess) return e;
        for (int l = 0; l < n; ++l) {
            if ((e = cudaStreamWaitEvent(ls[l], ev[kMaxLat], 0)) != cudaSuccess) return e;
            if ((e = f(l, ls[l])) != cudaSuccess) return e;
            if ((e = cudaEventRecord(ev[l], ls[l])) != cudaSuccess) return e;
        }
        for (int l = 0; l < n; ++l)
            if ((e = cudaStreamWaitEvent(cs, ev[l], 0)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    template <class S, class IL>
    cudaError_t build(S* sv, int n_, const IL& il) {
        constexpr cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
        n = n_;
        LatCtlArgs ca{};
        LatLoopArgs la{};
        ca.n = la.n = n;
        la.together = 1;
        for (int l = 0; l < n; ++l) ca.st[l] = la.st[l] = sv[l].dstate;
        cudaError_t e, le;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return e;
        for (int l = 0; l < n; ++l)
            if ((e = cudaStreamCreateWithFlags(&ls[l], cudaStreamNonBlocking)) != cudaSuccess) return e;
        for (int l = 0; l <= kMaxLat; ++l)
            if ((e = cudaEventCreateWithFlags(&ev[l], cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess) return e;
        cudaGraphConditionalHandle outer, inner, run[kMaxLat];
        if ((e = cudaGraphConditionalHandleCreate(&outer, graph, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
            return e;
        if ((e = cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, mode)) != cudaSuccess) return e;
        lat_first_kernel<<<1, 32, 0, cs>>>(ca, outer);
        le = cudaGetLastError();
        cudaGraph_t round = nullptr, body = nullptr, tail[kMaxLat] = {};
        if (le == cudaSuccess) le = capture_conditional(cs, outer, cudaGraphCondTypeWhile, &round);
        e = cudaStreamEndCapture(cs, &graph);
        if (le != cudaSuccess) return le;
        if (e != cudaSuccess) return e;
        // one round of cycles: the lattices' restarts side by side, the inner loop, then each
        // lattice's reliable update (if its solution moved) side by side
        if ((e = cudaGraphConditionalHandleCreate(&inner, round, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
            return e;
        for (int l = 0; l < n; ++l)
            if ((e = cudaGraphConditionalHandleCreate(&run[l], round, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
                return e;
        if ((e = cudaStreamBeginCaptureToGraph(cs, round, nullptr, nullptr, 0, mode)) != cudaSuccess) return e;
        ctl_arm_kernel<<<1, 32, 0, cs>>>(inner);
        le = cudaGetLastError();
        if (le == cudaSuccess)
            le = branches([&](int l, cudaStream_t s) { return sv[l].launch_restart(s, true); });
        if (le == cudaSuccess) {
            lattice_loop_base<<<1, 32, 0, cs>>>(la);
            le = cudaGetLastError();
        }
        if (le == cudaSuccess) le = capture_conditional(cs, inner, cudaGraphCondTypeWhile, &body);
        if (le == cudaSuccess)
            le = branches([&](int l, cudaStream_t s) {
                lat_mid_kernel<<<1, 32, 0, s>>>(sv[l].dstate, run[l]);
                cudaError_t r = cudaGetLastError();
                return r == cudaSuccess ? capture_conditional(s, run[l], cudaGraphCondTypeIf, &tail[l]) : r;
            });
        if (le == cudaSuccess) {
            lat_decide_kernel<<<1, 32, 0, cs>>>(ca, outer);
            le = cudaGetLastError();
        }
        e = cudaStreamEndCapture(cs, &round);
        if (le != cudaSuccess) return le;
        if (e != cudaSuccess) return e;
        // one iteration of every lattice (side by side) and the loop test
        if ((e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, mode)) != cudaSuccess) return e;
        le = branches([&](int l, cudaStream_t s) { return il.iteration_of(l, s); });
        if (le == cudaSuccess) {
            lattice_loop_cond<<<1, 32, 0, cs>>>(inner, la);
            le = cudaGetLastError();
        }
        e = cudaStreamEndCapture(cs, &body);
        if (le != cudaSuccess) return le;
        if (e != cudaSuccess) return e;
        // each lattice's reliable update
        for (int l = 0; l < n; ++l) {
            if ((e = cudaStreamBeginCaptureToGraph(cs, tail[l], nullptr, nullptr, 0, mode)) != cudaSuccess) return e;
            le = sv[l].launch_tail(cs);
            if (le == cudaSuccess) {
                lat_end_kernel<<<1, 32, 0, cs>>>(sv[l].dstate);
                le = cudaGetLastError();
            }
            e = cudaStreamEndCapture(cs, &tail[l]);
            if (le != cudaSuccess) return le;
            if (e != cudaSuccess) return e;
        }
        return cudaGraphInstantiate(&exec, graph, 0);
    }
};

// Runs every cycle of the batch in one LatticeSolveGraph launch; false (nothing launched)
// if the graph cannot be built here, and the host then drives the rounds.
template <class S, class IL>
bool lattice_device_cycles(S* sv, int n, const IL& il, cudaStream_t st, int* r) {
    NvtxRange nvtx("lq lattices: cycles (one graph)");
    int counted[kMaxLat];
    for (int l = 0; l < n; ++l) counted[l] = sv[l].launches;
    LatticeSolveGraph lg;
    cudaError_t e = lg.build(sv, n, il);
    for (int l = 0; l < n; ++l) sv[l].launches = counted[l];   // the builders counted while captured
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    *r = LQ_OK;
    for (int l = 0; l < n && e == cudaSuccess; ++l) e = sv[l].upload_ctl();
    if (e == cudaSuccess) e = cudaGraphLaunch(lg.exec, st);
    for (int l = 0; l < n && e == cudaSuccess; ++l) e = sv[l].read_state_async();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        *r = cuda_fail(e, "lattice solve graph");
        return true;
    }
    for (int l = 0; l < n; ++l) {
        sv[l].hc = sv[l].hs.ctl;
        sv[l].launches += sv[l].hc.launches;
        sv[l].k_max = sv[l].hc.k_max;
    }
    return true;
}

template <int IP, int IF, int IL, int HP, int IBS>
int run_lattices_bs(int n, const LatticeJob* jobs, const lq_cg_params& prm, double delta, char* ws,
                    lq_cg_info* info, cudaStream_t st) {
    using S = Solve<IP, IF, IL, HP, IBS>;
    std::unique_ptr<S[]> sv(new S[n]);
    int64_t sites = 0;
    for (int l = 0; l < n; ++l) {
        const LatticeJob& j = jobs[l];
        sv[l].init(j.g, j.m_q, j.nb, j.U, j.eta, j.x, prm, delta, j.w, ws + j.off, st);
        sites += (int64_t)j.g.V * j.nb;
    }
    const int chunk = prm.chunk > 0 ? prm.chunk : (sites >= (1 << 18) ? 8 : 32);
    int r;
    for (int l = 0; l < n; ++l)
        if ((r = sv[l].begin()) != LQ_OK) return r;

    InnerLaunches<S> il;
    il.build(sv.get(), n);
    const bool use_graph = (prm.flags & LQ_CG_NO_GRAPH) == 0;
    cudaError_t e;
    // device-driven loop (one graph launch until a lattice's cycle ends); if the conditional
    // graph cannot be built, chunks of iterations captured as a plain graph
    LoopGraph lg;
    bool device_loop = false;
    // reliable updates of all lattices taken together (one host round trip per round of
    // cycles), unless each lattice is to take its own as soon as its inner loop stops
    const bool together = (prm.flags & LQ_CG_LATTICE_OWN_CYCLES) == 0;
    if (use_graph) {
        LatLoopArgs la{};
        la.n = n;
        la.together = together ? 1 : 0;
        for (int l = 0; l < n; ++l) la.st[l] = sv[l].dstate;
        if (lg.build(il, la) == cudaSuccess) {
            device_loop = true;
        } else {
            (void)cudaGetLastError();
            lg.reset();
        }
    }
    ChunkGraph cg;
    if (use_graph && !device_loop && (e = cg.capture(il, chunk)) != cudaSuccess)
        return cuda_fail(e, "inner-loop graph capture");

    // every round of cycles in one graph launch when the rounds are taken together
    bool on_device = false;
    if (device_loop && together) {
        on_device = lattice_device_cycles(sv.get(), n, il, st, &r);
        if (on_device && r != LQ_OK) return r;
    }
    bool in_cycle[kMaxLat] = {}, finished[kMaxLat] = {};
    int chunks = 0;
    while (!on_device) {
        bool any = false;
        for (int l = 0; l < n; ++l) {
            if (!in_cycle[l] && !finished[l]) {
                if (sv[l].plan()) {
                    if ((r = sv[l].start_cycle()) != LQ_OK) return r;
                    in_cycle[l] = true;
                } else {
                    finished[l] = true;
                }
            }
            any |= in_cycle[l];
        }
        if (!any) break;
        NvtxRange nvtx("lq lattices: inner CG of every running lattice");
        if (device_loop) {
            if ((e = cudaGraphLaunch(lg.exec, st)) != cudaSuccess) return cuda_fail(e, "inner-loop graph");
        } else if (use_graph) {
            if ((e = cudaGraphLaunch(cg.exec, st)) != cudaSuccess) return cuda_fail(e, "inner-loop graph");
        } else {
            for (int j = 0; j < chunk; ++j)
                if ((e = il.iteration(st)) != cudaSuccess) return cuda_fail(e, "inner loop");
        }
        ++chunks;
        for (int l = 0; l < n; ++l)
            if ((in_cycle[l] || (device_loop && l == 0)) && (e = sv[l].read_state_async()) != cudaSuccess)
                return cuda_fail(e, "inner loop");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "inner loop");
        // launches each lattice took part in: the iterations (and, for the device loop, the
        // prologue and one condition kernel per trip)
        const int trips = device_loop ? sv[0].hs.loop_trips : chunk;
        for (int l = 0; l < n; ++l) sv[l].launches += device_loop ? 4 * trips + 1 : 3 * chunk;
        bool ended[kMaxLat] = {};
        int n_in = 0, n_ended = 0;
        for (int l = 0; l < n; ++l) {
            if (!in_cycle[l]) continue;
            ++n_in;
            // iterations launched in this lattice's cycle; K2 stops every right-hand side at
            // k_max, so this guard never decides
            sv[l].guard += trips;
            ended[l] = sv[l].hs.all_stop || sv[l].guard > sv[l].k_max + 2 * (device_loop ? 1 : chunk);
            n_ended += ended[l] ? 1 : 0;
        }
        if (n_ended == 0 || (together && n_ended < n_in)) continue;
        // the ended lattices' reliable updates: solution updates and outer residuals enqueued
        // for all of them, one read-back of their state records, then each one's outcome
        for (int l = 0; l < n; ++l)
            if (ended[l] && (r = sv[l].end_cycle_launch()) != LQ_OK) return r;
        for (int l = 0; l < n; ++l)
            if (ended[l] && (e = sv[l].read_state_async()) != cudaSuccess) return cuda_fail(e, "residual");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "residual");
        for (int l = 0; l < n; ++l) {
            if (!ended[l]) continue;
            sv[l].end_cycle_collect();
            in_cycle[l] = false;
        }
    }
    int worst = LQ_OK, at = 0;
    for (int l = 0; l < n; ++l) {
        const int s = sv[l].finish(info ? info + at : nullptr);
        at += jobs[l].nb;
        if (s < 0 && (worst >= 0 || s < worst)) worst = s;
        if (s == LQ_NOT_CONVERGED && worst == LQ_OK) worst = LQ_NOT_CONVERGED;
    }
    return worst;
}

// Mean device time of the all-lattice K1 launch with block size IBS, on a p filled with a
// small constant (every state slot running, so every block works); ms, or < 0 on error.
template <int IP, int IF, int IL, int HP, int IBS>
double time_k1(int n, const LatticeJob* jobs, char* ws, cudaStream_t st) {
    using S = Solve<IP, IF, IL, HP, IBS>;
    std::unique_ptr<S[]> sv(new S[n]);
    lq_cg_params prm{};
    prm.tol = 1e-10;
    prm.max_iter = 1;
    for (int l = 0; l < n; ++l) {
        const LatticeJob& j = jobs[l];
        sv[l].init(j.g, j.m_q, j.nb, j.U, j.eta, j.x, prm, 0.0, j.w, ws + j.off, st);
        if (cudaMemsetAsync(sv[l].dstate, 0, sizeof(SolverState), st) != cudaSuccess ||
            cudaMemsetAsync(ws + j.off + j.w.p, 0x3c, spinor_bytes((int64_t)j.g.V * j.nb, IP), st) != cudaSuccess)
            return -1.0;
        if constexpr (IP != LQ_F64 && IP != LQ_F64X) {
            if (convert_gauge(j.g, LQ_F64, LQ_LAYOUT_LEX, j.U, IP, IF, IL, ws + j.off + j.w.u_low, st) != cudaSuccess)
                return -1.0;
        } else if constexpr (IP == LQ_F64X) {
            if (convert_gauge(j.g, LQ_F64, LQ_LAYOUT_LEX, j.U, LQ_F64X, 18, LQ_LAYOUT_EO, ws + j.off + j.w.u_x, st) !=
                cudaSuccess)
                return -1.0;
        }
    }
    InnerLaunches<S> il;
    il.build(sv.get(), n);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
    constexpr int kWarm = 2, kReps = 6;
    bool ok = true;
    for (int i = 0; i < kWarm; ++i) ok &= il.k1_only(st) == cudaSuccess;
    ok &= cudaEventRecord(e0, st) == cudaSuccess;
    for (int i = 0; i < kReps; ++i) ok &= il.k1_only(st) == cudaSuccess;
    ok &= cudaEventRecord(e1, st) == cudaSuccess;
    ok &= cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0.f;
    ok &= cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok ? ms / kReps : -1.0;
}

// the tuning cache (lattices.cu)
bool tune_lookup(const std::string& key, int* block);
void tune_store(const std::string& key, int block);
std::string tune_key(int mode, int n, const LatticeJob* jobs);

constexpr int kTuneBlocks[3] = {64, 128, 256};

template <int IP, int IF, int IL, int HP>
int run_lattices(int mode, int n, const LatticeJob* jobs, const lq_cg_params& prm, double delta, char* ws,
                 lq_cg_info* info, cudaStream_t st) {
    int bs = kBS;
    if (prm.flags & LQ_CG_BLOCK_64) {
        bs = 64;
    } else if (prm.flags & LQ_CG_BLOCK_128) {
        bs = 128;
    } else if (prm.flags & LQ_CG_BLOCK_256) {
        bs = 256;
    } else if (prm.flags & LQ_CG_AUTOTUNE) {
        const std::string key = tune_key(mode, n, jobs);
        if (!tune_lookup(key, &bs)) {
            const double t[3] = {time_k1<IP, IF, IL, HP, 64>(n, jobs, ws, st),
                                 time_k1<IP, IF, IL, HP, 128>(n, jobs, ws, st),
                                 time_k1<IP, IF, IL, HP, 256>(n, jobs, ws, st)};
            int best = -1;
            for (int i = 0; i < 3; ++i)
                if (t[i] >= 0.0 && (best < 0 || t[i] < t[best])) best = i;
            if (best < 0) return fail(LQ_ERR_CUDA, "block-size tuning failed: %s", cudaGetErrorString(cudaGetLastError()));
            bs = kTuneBlocks[best];
            tune_store(key, bs);
        }
    }
    switch (bs) {
        case 64: return run_lattices_bs<IP, IF, IL, HP, 64>(n, jobs, prm, delta, ws, info, st);
        case 256: return run_lattices_bs<IP, IF, IL, HP, 256>(n, jobs, prm, delta, ws, info, st);
        default: return run_lattices_bs<IP, IF, IL, HP, 128>(n, jobs, prm, delta, ws, info, st);
    }
}

// per-mode instantiations (solver_lat_*.cu)
int lattices_f64(int n, const LatticeJob* jobs, const lq_cg_params& prm, double delta, char* ws, lq_cg_info* info,
                 cudaStream_t st);
int lattices_f64x(int n, const LatticeJob* jobs, const lq_cg_params& prm, double delta, char* ws, lq_cg_info* info,
                  cudaStream_t st);
int lattices_mixed_f32(int n, const LatticeJob* jobs, const lq_cg_params& prm, double delta, char* ws,
                       lq_cg_info* info, cudaStream_t st);
int lattices_mixed_f16(int n, const LatticeJob* jobs, const lq_cg_params& prm, double delta, char* ws,
                       lq_cg_info* info, cudaStream_t st);

}  // namespace solver_detail

}  // namespace lq
