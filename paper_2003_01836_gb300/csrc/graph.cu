// graph.cu -- a solve captured once and replayed as one CUDA graph.
//
// Fixed positions.  Algorithm 1's setup depends only on the positions: the trees (Sec. II-D),
// the interaction lists (Eq. 13) and the work plans of the upward pass and the sweep.  The
// arithmetic that depends on the charges is the upward pass (Eq. 12) and the sweep (Eq. 9, 11).
// Iterative methods apply the same particle interaction to a new charge vector at every step
// (the treecode as a matrix-vector product), so bltc_graph_create builds the setup once,
// allocates every buffer a replay needs, and captures the charge-dependent launches:
//   gather of q into tree order -> leaf sums and M2M levels -> sweep -> finalize into phi.
//
// New positions at every launch.  bltc_graph_create_positions captures the whole of Algorithm 1
// (tree, lists, upward pass, plan, sweep, finalize) sized on the device: capacities from a first
// solve with some headroom, every count kept in device memory, kernels launched over the
// capacities (Caps in internal.cuh).  The capture allocates nothing: a first pass of the sized
// solve runs uncaptured and measures what it allocates, and the captured pass takes the same
// buffers from one arena of that size.  A launch is one cudaGraphLaunch and one read of the
// overflow flag; a solve that exceeded a capacity is redone on the host-driven path, and the
// graph is rebuilt for the new sizes.
#include <algorithm>
#include <cmath>
#include <memory>

#include "internal.cuh"

namespace bltc {
namespace {

__global__ void k_gather_q(const double* __restrict__ q, const int32_t* __restrict__ perm, int64_t n,
                           double* __restrict__ pq) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) pq[i] = q[perm[i]];
}

}  // namespace

// The objects of one solve (trees, lists, upward plan, sweep buffers).
struct SolveObjects {
    Tree st;
    std::unique_ptr<Tree> btp;
    const Tree* bt = nullptr;
    Lists L;
    UpwardPlan up;
    SweepBuffers sb;
};

struct GraphSolve {
    Context* c = nullptr;
    bltc_params p{};
    int64_t n = 0;
    const double *x = nullptr, *y = nullptr, *z = nullptr;
    const double* q = nullptr;
    double* phi = nullptr;
    bool positions = false;
    double headroom = 1.25;
    Caps caps_s, caps_b;                  // source tree, lists and plans; batch tree
    DBuf<int32_t> flag;                   // the overflow flag of the sized solve
    int32_t* flag_host = nullptr;         // pinned: its value after the last launch
    DBuf<char> arena;                     // every buffer of the captured sized solve
    std::unique_ptr<SolveObjects> o;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;                  // kernels one replay launches
    int64_t launches = 0, redone = 0, captures = 0;
    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }
    ~GraphSolve() {
        drop_graph();
        o.reset();                        // arena buffers are not freed one by one
        if (flag_host) cudaFreeHost(flag_host);
    }
};

namespace {

// Runs `body` as a capture on a private stream, with no allocation allowed outside the
// context's arena, and instantiates the graph.
template <typename F>
void capture(Context* c, GraphSolve* g, F body) {
    cudaStream_t cs = nullptr;
    BLTC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t user = c->stream;
    const bool timing = c->timing;
    const int64_t launches0 = c->launches;
    c->stream = cs;
    c->timing = false;
    c->capturing = true;
    auto restore = [&] {
        c->stream = user;
        c->timing = timing;
        c->capturing = false;
        c->launches = launches0;
        c->arena = Context::Arena();
    };
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        restore();
        cudaStreamDestroy(cs);
        throw Error(BLTC_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    }
    try {
        body(cs);
    } catch (...) {
        cudaGraph_t partial = nullptr;
        cudaStreamEndCapture(cs, &partial);
        if (partial) cudaGraphDestroy(partial);
        restore();
        cudaStreamDestroy(cs);
        throw;
    }
    g->kernels = c->launches - launches0;
    e = cudaStreamEndCapture(cs, &g->graph);
    restore();
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) throw Error(BLTC_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    BLTC_CUDA(cudaGraphInstantiate(&g->exec, g->graph, 0));
    ++g->captures;
}

// The solve sized on the device: the same steps as the host-driven solve, every count in
// device memory, no host synchronisation.
void run_sized(GraphSolve* g, SolveObjects* o) {
    Context* c = g->c;
    const bltc_params& p = g->p;
    build_tree(c, g->x, g->y, g->z, g->q, g->n, p.leaf_size, &o->st, &g->caps_s);
    o->bt = &o->st;
    if (p.batch_size != p.leaf_size) {
        o->btp.reset(new Tree());
        build_tree(c, g->x, g->y, g->z, nullptr, g->n, p.batch_size, o->btp.get(), &g->caps_b);
        o->bt = o->btp.get();
    }
    build_lists(c, o->bt, &o->st, p.theta, p.degree, &o->L, &g->caps_s);
    prepare_upward(c, &o->st, &o->L, p.degree, p.precision, &o->up);
    // the upward pass's kernels on a second branch, beside the work plan (both follow the
    // lists and are independent); captured, the fork and the join become graph edges
    c->fork();
    cudaStream_t main_stream = c->stream;
    c->stream = c->side;
    try {
        run_upward(c, &o->st, o->up);
    } catch (...) {
        c->stream = main_stream;
        c->join();
        throw;
    }
    c->stream = main_stream;
    try {
        prepare_plan(c, &o->L, p.degree, p.precision, p.tile);
        alloc_sweep_buffers(c, &o->L, &o->sb);
    } catch (...) {
        c->join();
        throw;
    }
    c->join();
    run_sweep(c, &o->L, o->bt, &o->st, p, g->phi, o->sb);
}

// A host-driven solve of the bound positions and charges into phi, whose counts with the
// graph's headroom become the capacities.
void size_from_solve(GraphSolve* g) {
    Context* c = g->c;
    const bltc_params& p = g->p;
    SolveObjects o;
    build_tree(c, g->x, g->y, g->z, g->q, g->n, p.leaf_size, &o.st);
    o.bt = &o.st;
    if (p.batch_size != p.leaf_size) {
        o.btp.reset(new Tree());
        build_tree(c, g->x, g->y, g->z, nullptr, g->n, p.batch_size, o.btp.get());
        o.bt = o.btp.get();
    }
    build_lists(c, o.bt, &o.st, p.theta, p.degree, &o.L);
    prepare_upward(c, &o.st, &o.L, p.degree, p.precision, &o.up);
    run_upward(c, &o.st, o.up);
    evaluate(c, &o.L, o.bt, &o.st, p, g->phi);
    Caps s, b;
    tree_counts(c, o.st, &s);
    if (o.btp) tree_counts(c, *o.btp, &b);
    s.app = o.L.n_app;
    s.dir = o.L.n_dir;
    s.slots = o.up.n_slots;
    s.up_items = o.up.n_items;
    s.m2m = o.up.h.empty() ? 0 : *std::max_element(o.up.h.begin(), o.up.h.end());
    s.items = o.L.plan.n_items;
    s.partial_len = o.L.plan.partial_len;
    s.mpart_len = o.L.plan.mpart_len;
    const double h = g->headroom;
    auto grow = [h](int64_t v, int64_t add) { return static_cast<int64_t>(std::ceil(static_cast<double>(v) * h)) + add; };
    auto grow32 = [&](int64_t v, int64_t add) {
        return static_cast<int32_t>(std::min<int64_t>(grow(v, add), int64_t(1) << 30));
    };
    auto tree_caps = [&](Caps& t) {
        t.nodes = grow32(t.nodes, 64);
        t.levels += 2;
        t.level_nodes = std::min(t.nodes, grow32(t.level_nodes, 64));
        t.chunks = grow(t.chunks, 64);
        t.flag = g->flag.p;
    };
    tree_caps(s);
    if (o.btp) tree_caps(b);
    s.app = grow(s.app, 1024);
    s.dir = grow(s.dir, 1024);
    s.slots = grow32(s.slots, 64);
    s.up_items = grow32(s.up_items, 64);
    s.m2m = grow32(s.m2m, 16);
    s.items = grow(s.items, 1024);
    s.partial_len = grow(s.partial_len, g->n);
    s.mpart_len = grow(s.mpart_len, g->n);
    g->caps_s = s;
    g->caps_b = b;
}

// Measures the sized solve's allocations (one uncaptured run, which also checks that the
// capacities hold), then captures it on an arena of that size.
void build_positions_graph(GraphSolve* g) {
    Context* c = g->c;
    g->drop_graph();
    g->o.reset();
    g->arena = DBuf<char>();
    BLTC_CUDA(cudaMemsetAsync(g->flag.p, 0, sizeof(int32_t), c->stream));
    c->arena = Context::Arena();
    c->arena.measure = true;
    try {
        SolveObjects probe;
        run_sized(g, &probe);
    } catch (...) {
        c->arena = Context::Arena();
        throw;
    }
    const size_t bytes = c->arena.measured;
    c->arena = Context::Arena();
    const int32_t f = *reinterpret_cast<const int32_t*>(c->read_words(g->flag.p, 1));
    if (f != 0) throw Error(BLTC_ERR_STATE, "graph: the sized solve exceeded capacities taken from the same positions");
    g->arena = DBuf<char>(c, static_cast<int64_t>(bytes));
    BLTC_CUDA(cudaStreamSynchronize(c->stream));     // the arena is allocated before the capture reads it
    g->o.reset(new SolveObjects());
    capture(c, g, [&](cudaStream_t cs) {
        c->arena.base = g->arena.p;
        c->arena.size = bytes;
        BLTC_CUDA(cudaMemsetAsync(g->flag.p, 0, sizeof(int32_t), cs));
        run_sized(g, g->o.get());
        BLTC_CUDA(cudaMemcpyAsync(g->flag_host, g->flag.p, sizeof(int32_t), cudaMemcpyDeviceToHost, cs));
    });
}

}  // namespace

GraphSolve* graph_create(Context* c, const double* x, const double* y, const double* z, const double* q,
                         int64_t n, const bltc_params& p, double* phi) {
    std::unique_ptr<GraphSolve> g(new GraphSolve());
    g->c = c;
    g->p = p;
    g->n = n;
    g->q = q;
    g->phi = phi;
    g->o.reset(new SolveObjects());
    SolveObjects& o = *g->o;
    build_tree(c, x, y, z, q, n, p.leaf_size, &o.st);
    o.bt = &o.st;
    if (p.batch_size != p.leaf_size) {
        o.btp.reset(new Tree());
        build_tree(c, x, y, z, nullptr, n, p.batch_size, o.btp.get());
        o.bt = o.btp.get();
    }
    build_lists(c, o.bt, &o.st, p.theta, p.degree, &o.L);
    prepare_upward(c, &o.st, &o.L, p.degree, p.precision, &o.up);
    // one plain solve: validates the arguments, builds the sweep's work plan, and loads and
    // configures every kernel before the capture
    run_upward(c, &o.st, o.up);
    evaluate(c, &o.L, o.bt, &o.st, p, phi);
    alloc_sweep_buffers(c, &o.L, &o.sb);
    BLTC_CUDA(cudaStreamSynchronize(c->stream));
    capture(c, g.get(), [&](cudaStream_t cs) {
        if (n > 0) {
            k_gather_q<<<grid_for(n, 256), 256, 0, cs>>>(q, o.st.perm.p, n, o.st.pq.p); ++c->launches;
            BLTC_LAUNCH_CHECK("gather charges");
        }
        run_upward(c, &o.st, o.up);
        run_sweep(c, &o.L, o.bt, &o.st, p, phi, o.sb);
    });
    return g.release();
}

GraphSolve* graph_create_positions(Context* c, const double* x, const double* y, const double* z,
                                   const double* q, int64_t n, const bltc_params& p, double* phi,
                                   double headroom) {
    require(headroom == 0.0 || (std::isfinite(headroom) && headroom >= 1.0 && headroom <= 16.0),
            "graph: headroom must be 0 (default) or in [1, 16]");
    std::unique_ptr<GraphSolve> g(new GraphSolve());
    g->c = c;
    g->p = p;
    g->n = n;
    g->x = x;
    g->y = y;
    g->z = z;
    g->q = q;
    g->phi = phi;
    g->positions = true;
    if (headroom > 0.0) g->headroom = headroom;
    g->flag = DBuf<int32_t>(c, 1);
    BLTC_CUDA(cudaMallocHost(&g->flag_host, 16));
    *g->flag_host = 0;
    size_from_solve(g.get());
    build_positions_graph(g.get());
    return g.release();
}

void graph_launch(Context* c, GraphSolve* g) {
    if (g->c != c) throw Error(BLTC_ERR_STATE, "graph: launched on another context");
    c->mark(Context::kStart);
    BLTC_CUDA(cudaGraphLaunch(g->exec, c->stream));
    c->launches += g->kernels;
    c->mark(Context::kEnd);
    ++g->launches;
    if (!g->positions) return;
    BLTC_CUDA(cudaStreamSynchronize(c->stream));
    if (*g->flag_host == 0) return;
    // A capacity was exceeded (or the input is not finite): solve on the host-driven path, which
    // reports bad input, and rebuild the graph for these positions' sizes.
    ++g->redone;
    size_from_solve(g);
    build_positions_graph(g);
}

int64_t graph_kernels(const GraphSolve* g) { return g->kernels; }

void graph_info(const GraphSolve* g, int64_t out[4]) {
    out[0] = g->kernels;
    out[1] = g->launches;
    out[2] = g->redone;
    out[3] = g->captures;
}

void graph_destroy(GraphSolve* g) { delete g; }

}  // namespace bltc
