// graph.cu -- a solve with fixed positions, captured once and replayed as one CUDA graph.
//
// Algorithm 1's setup depends only on the positions: the trees (Sec. II-D), the interaction
// lists (Eq. 13) and the work plans of the upward pass and the sweep.  The arithmetic that
// depends on the charges is the upward pass (Eq. 12) and the sweep (Eq. 9, 11).  Iterative
// methods apply the same particle interaction to a new charge vector at every step (the
// treecode as a matrix-vector product), so this module builds the setup once, allocates every
// buffer a replay needs, and captures the charge-dependent launches on a private stream:
//   gather of q into tree order -> leaf sums and M2M levels -> sweep -> finalize into phi.
// A replay is one cudaGraphLaunch: no host synchronisation, no allocation, no per-kernel
// launch overhead.
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

struct GraphSolve {
    Context* c = nullptr;
    bltc_params p{};
    int64_t n = 0;
    const double* q = nullptr;
    double* phi = nullptr;
    Tree st;
    std::unique_ptr<Tree> btp;
    const Tree* bt = nullptr;
    Lists L;
    UpwardPlan up;
    SweepBuffers sb;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;                  // kernels one replay launches
    ~GraphSolve() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
    }
};

GraphSolve* graph_create(Context* c, const double* x, const double* y, const double* z, const double* q,
                         int64_t n, const bltc_params& p, double* phi) {
    std::unique_ptr<GraphSolve> g(new GraphSolve());
    g->c = c;
    g->p = p;
    g->n = n;
    g->q = q;
    g->phi = phi;
    build_tree(c, x, y, z, q, n, p.leaf_size, &g->st);
    g->bt = &g->st;
    if (p.batch_size != p.leaf_size) {
        g->btp.reset(new Tree());
        build_tree(c, x, y, z, nullptr, n, p.batch_size, g->btp.get());
        g->bt = g->btp.get();
    }
    build_lists(c, g->bt, &g->st, p.theta, p.degree, &g->L);
    prepare_upward(c, &g->st, &g->L, p.degree, p.precision, &g->up);
    // one plain solve: validates the arguments, builds the sweep's work plan, and loads and
    // configures every kernel before the capture
    run_upward(c, &g->st, g->up);
    evaluate(c, &g->L, g->bt, &g->st, p, phi);
    alloc_sweep_buffers(c, &g->L, &g->sb);
    BLTC_CUDA(cudaStreamSynchronize(c->stream));

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
    };
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        restore();
        cudaStreamDestroy(cs);
        throw Error(BLTC_ERR_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
    }
    try {
        if (n > 0) {
            k_gather_q<<<grid_for(n, 256), 256, 0, cs>>>(q, g->st.perm.p, n, g->st.pq.p); ++c->launches;
            BLTC_LAUNCH_CHECK("gather charges");
        }
        run_upward(c, &g->st, g->up);
        run_sweep(c, &g->L, g->bt, &g->st, p, phi, g->sb);
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
    return g.release();
}

void graph_launch(Context* c, GraphSolve* g) {
    if (g->c != c) throw Error(BLTC_ERR_STATE, "graph: launched on another context");
    c->mark(Context::kStart);
    BLTC_CUDA(cudaGraphLaunch(g->exec, c->stream));
    c->launches += g->kernels;
    c->mark(Context::kEnd);
}

int64_t graph_kernels(const GraphSolve* g) { return g->kernels; }

void graph_destroy(GraphSolve* g) { delete g; }

}  // namespace bltc
