// api.cu -- the extern "C" boundary declared in include/bltc.h: argument checks, status
// codes, the context (device, stream, allocator, Chebyshev tables) and the composition of
// the steps into Algorithm 1 (bltc_solve).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <tuple>
#include <vector>

#include "internal.cuh"

struct bltc_context {
    bltc::Context c;
    // autotuner cache: (log2 n, degree, kernel, precision, theta * 1000, distribution shape)
    // -> (leaf, batch)
    std::map<std::tuple<int, int, int, int, int, int>, std::pair<int32_t, int32_t>> tuned;
    // tile cache: the same key plus (leaf, batch) -> params.tile
    std::map<std::tuple<int, int, int, int, int, int, int32_t, int32_t>, int32_t> tuned_tile;
};
struct bltc_tree {
    bltc::Tree t;
};
struct bltc_lists {
    bltc::Lists l;
};
struct bltc_graph {
    bltc::GraphSolve* g = nullptr;
    bltc_context* ctx = nullptr;
};

namespace bltc {

void* Context::dalloc(size_t bytes) {
    void* p = nullptr;
    if (arena.base) {
        const size_t b = Arena::footprint(bytes);
        if (arena.used + b > arena.size) throw Error(BLTC_ERR_STATE, "graph arena exhausted");
        p = arena.base + arena.used;
        arena.used += b;
        return p;
    }
    if (capturing) throw Error(BLTC_ERR_STATE, "device allocation inside a graph capture");
    if (arena.measure) arena.measured += Arena::footprint(bytes);
    if (alloc_fn) {
        p = alloc_fn(bytes, stream, alloc_user);
        if (!p) throw Error(BLTC_ERR_OOM, "allocator returned NULL for " + std::to_string(bytes) + " bytes");
        return p;
    }
    cudaError_t e = cudaMallocFromPoolAsync(&p, bytes, pool, stream);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        throw Error(BLTC_ERR_OOM, "device pool out of memory for " + std::to_string(bytes) + " bytes");
    }
    if (e != cudaSuccess) throw Error(BLTC_ERR_CUDA, std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e));
    return p;
}

void Context::dfree(void* p, size_t bytes) {
    if (!p) return;
    if (free_fn) {
        free_fn(p, bytes, stream, alloc_user);
        return;
    }
    cudaFreeAsync(p, stream);
}

void Context::fork() {
    if (!side) {
        BLTC_CUDA(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
        BLTC_CUDA(cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming));
        BLTC_CUDA(cudaEventCreateWithFlags(&join_ev, cudaEventDisableTiming));
    }
    BLTC_CUDA(cudaEventRecord(fork_ev, stream));
    BLTC_CUDA(cudaStreamWaitEvent(side, fork_ev, 0));
}

void Context::join() {
    BLTC_CUDA(cudaEventRecord(join_ev, side));
    BLTC_CUDA(cudaStreamWaitEvent(stream, join_ev, 0));
}

const int64_t* Context::read_words(const void* dev, int words) {
    if (words > kPinnedWords) throw Error(BLTC_ERR_ARG, "read_words: too many words");
    BLTC_CUDA(cudaMemcpyAsync(pinned, dev, sizeof(int64_t) * words, cudaMemcpyDeviceToHost, stream));
    BLTC_CUDA(cudaStreamSynchronize(stream));
    return pinned;
}

// t_k = cos(pi k / n), k = 0..n (Eq. 6), generated on the host in FP64 and uploaded once.
const double* Context::cheb_table(int degree) {
    if (degree < 1 || degree > BLTC_MAX_DEGREE) throw Error(BLTC_ERR_ARG, "degree out of range");
    if (!cheb_t[degree]) {
        double h[BLTC_MAX_DEGREE + 1];
        const double pi = 3.14159265358979323846;
        for (int k = 0; k <= degree; ++k) h[k] = std::cos(pi * static_cast<double>(k) / static_cast<double>(degree));
        double* d = nullptr;
        BLTC_CUDA(cudaMalloc(&d, sizeof(double) * (degree + 1)));
        BLTC_CUDA(cudaMemcpy(d, h, sizeof(double) * (degree + 1), cudaMemcpyHostToDevice));
        cheb_t[degree] = d;
    }
    return cheb_t[degree];
}

static void check_params(const bltc_params* p) {
    require(p != nullptr, "params is NULL");
    require(p->degree >= 1 && p->degree <= BLTC_MAX_DEGREE, "degree must be in [1, 16]");
    require(std::isfinite(p->theta) && p->theta >= 0.0 && p->theta < 1.0,
            "theta must satisfy 0 <= theta < 1");
    require(p->leaf_size >= 1 && p->batch_size >= 1, "leaf_size and batch_size must be >= 1");
    require(p->kernel == BLTC_KERNEL_COULOMB || p->kernel == BLTC_KERNEL_YUKAWA ||
                p->kernel >= BLTC_KERNEL_USER_BASE,
            "unknown kernel");
    require(p->kernel != BLTC_KERNEL_YUKAWA || (std::isfinite(p->kappa) && p->kappa >= 0.0),
            "kappa must be finite and >= 0");
    require(p->kernel < BLTC_KERNEL_USER_BASE || std::isfinite(p->kappa),
            "a user kernel's parameter (kappa) must be finite");
    require(p->precision == BLTC_PRECISION_FP64 || p->precision == BLTC_PRECISION_MIXED,
            "unknown precision");
    require(tile_valid(p->tile), "params.tile: group cap 0, 1, 2, 4 or 8 (bits 0-3), items per block 0..255 (bits 4-11), other bits 0");
}

template <typename F>
static bltc_status guarded(bltc_context* ctx, F&& f) {
    try {
        if (ctx) {
            ctx->c.err.clear();
            BLTC_CUDA(cudaSetDevice(ctx->c.device));
        }
        f();
        return BLTC_OK;
    } catch (const Error& e) {
        if (ctx) ctx->c.err = e.what();
        return e.status;
    } catch (const std::bad_alloc&) {
        if (ctx) ctx->c.err = "host out of memory";
        return BLTC_ERR_OOM;
    } catch (const std::exception& e) {
        if (ctx) ctx->c.err = e.what();
        return BLTC_ERR_CUDA;
    }
}

// The upward pass (Eq. 12) and the sweep's work plan both follow the lists and are
// independent: the pass's kernels run on the side stream while the plan, whose steps wait on
// device counts, is built on the main stream.  The pass's scratch is freed on the main stream
// after the join, so no buffer is reused while the side stream may still read it.
static void upward_beside_plan(Context* c, Tree* st, Lists* L, const bltc_params& p) {
    UpwardPlan up;
    prepare_upward(c, st, L, p.degree, p.precision, &up);
    c->mark(Context::kUpward);
    c->fork();
    cudaStream_t main_stream = c->stream;
    c->stream = c->side;
    try {
        run_upward(c, st, up);
    } catch (...) {
        c->stream = main_stream;
        c->join();
        throw;
    }
    c->stream = main_stream;
    try {
        prepare_plan(c, L, p.degree, p.precision, p.tile);
    } catch (...) {
        c->join();
        throw;
    }
    c->join();
}

void solve_device(Context* c, const double* x, const double* y, const double* z,
                  const double* q, int64_t n, const bltc_params& p, double* phi) {
    c->mark(Context::kStart);
    Tree st;
    build_tree(c, x, y, z, q, n, p.leaf_size, &st);
    std::unique_ptr<Tree> btp;
    const Tree* bt = &st;
    if (p.batch_size != p.leaf_size) {
        btp.reset(new Tree());
        build_tree(c, x, y, z, nullptr, n, p.batch_size, btp.get());
        bt = btp.get();
    }
    c->mark(Context::kTrees);
    Lists L;
    build_lists(c, bt, &st, p.theta, p.degree, &L);
    c->mark(Context::kLists);
    upward_beside_plan(c, &st, &L, p);
    evaluate(c, &L, bt, &st, p, phi);
}

// Algorithm 1 for distinct target and source sets: the source tree (leaf_size, charges) and
// the batch tree of the targets (batch_size, no charges) are built separately.
static void solve_device_targets(Context* c, const double* tx, const double* ty, const double* tz,
                                 int64_t nt, const double* sx, const double* sy, const double* sz,
                                 const double* sq, int64_t ns, const bltc_params& p, double* phi) {
    c->mark(Context::kStart);
    Tree st, bt;
    build_tree(c, sx, sy, sz, sq, ns, p.leaf_size, &st);
    build_tree(c, tx, ty, tz, nullptr, nt, p.batch_size, &bt);
    c->mark(Context::kTrees);
    Lists L;
    build_lists(c, &bt, &st, p.theta, p.degree, &L);
    c->mark(Context::kLists);
    upward_beside_plan(c, &st, &L, p);
    evaluate(c, &L, &bt, &st, p, phi);
}

}  // namespace bltc

using namespace bltc;

template <typename D, typename S>
static void copy_out(Context* c, D* host, const S* dev, int64_t count) {
    if (!host || count <= 0) return;
    if (sizeof(D) == sizeof(S)) {
        BLTC_CUDA(cudaMemcpyAsync(host, dev, sizeof(S) * count, cudaMemcpyDeviceToHost, c->stream));
        BLTC_CUDA(cudaStreamSynchronize(c->stream));
        return;
    }
    std::unique_ptr<S[]> tmp(new S[count]);
    BLTC_CUDA(cudaMemcpyAsync(tmp.get(), dev, sizeof(S) * count, cudaMemcpyDeviceToHost, c->stream));
    BLTC_CUDA(cudaStreamSynchronize(c->stream));
    for (int64_t i = 0; i < count; ++i) host[i] = static_cast<D>(tmp[i]);
}

extern "C" {

int bltc_version(void) { return BLTC_VERSION; }

bltc_status bltc_context_create(int device, void* stream, bltc_context** out) {
    if (!out) return BLTC_ERR_ARG;
    *out = nullptr;
    std::unique_ptr<bltc_context> ctx(new (std::nothrow) bltc_context());
    if (!ctx) return BLTC_ERR_OOM;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return BLTC_ERR_ARG;
    }
    Context& c = ctx->c;
    c.device = device;
    c.stream = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(device) != cudaSuccess) return BLTC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&c.sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return BLTC_ERR_CUDA;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c.pool, &props) != cudaSuccess) return BLTC_ERR_CUDA;
    uint64_t keep = ~0ULL;   // keep freed memory in the pool for the next call
    cudaMemPoolSetAttribute(c.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (cudaMallocHost(&c.pinned, sizeof(int64_t) * Context::kPinnedWords) != cudaSuccess) {
        cudaMemPoolDestroy(c.pool);
        return BLTC_ERR_CUDA;
    }
    *out = ctx.release();
    return BLTC_OK;
}

void bltc_context_destroy(bltc_context* ctx) {
    if (!ctx) return;
    Context& c = ctx->c;
    cudaSetDevice(c.device);
    cudaStreamSynchronize(c.stream);
    for (double*& t : c.cheb_t)
        if (t) cudaFree(t);
    for (cudaEvent_t& e : c.events)
        if (e) cudaEventDestroy(e);
    for (Context::UserKernel& k : c.user_kernels)
        if (k.lib) cudaLibraryUnload(k.lib);
    if (c.side) {
        cudaStreamSynchronize(c.side);
        cudaStreamDestroy(c.side);
    }
    if (c.fork_ev) cudaEventDestroy(c.fork_ev);
    if (c.join_ev) cudaEventDestroy(c.join_ev);
    if (c.pinned) cudaFreeHost(c.pinned);
    if (c.pool) cudaMemPoolDestroy(c.pool);
    delete ctx;
}

bltc_status bltc_context_set_stream(bltc_context* ctx, void* stream) {
    if (!ctx) return BLTC_ERR_ARG;
    ctx->c.stream = static_cast<cudaStream_t>(stream);
    return BLTC_OK;
}

bltc_status bltc_context_set_allocator(bltc_context* ctx, bltc_alloc_fn alloc, bltc_free_fn free_fn,
                                       void* user) {
    if (!ctx || (alloc == nullptr) != (free_fn == nullptr)) return BLTC_ERR_ARG;
    ctx->c.alloc_fn = alloc;
    ctx->c.free_fn = free_fn;
    ctx->c.alloc_user = user;
    return BLTC_OK;
}

bltc_status bltc_synchronize(bltc_context* ctx) {
    if (!ctx) return BLTC_ERR_ARG;
    return guarded(ctx, [&] { BLTC_CUDA(cudaStreamSynchronize(ctx->c.stream)); });
}

const char* bltc_last_error(const bltc_context* ctx) { return ctx ? ctx->c.err.c_str() : "no context"; }

int bltc_device_sm_count(const bltc_context* ctx) { return ctx ? ctx->c.sm_count : 0; }

int64_t bltc_context_launch_count(const bltc_context* ctx) { return ctx ? ctx->c.launches : -1; }

bltc_status bltc_context_set_timing(bltc_context* ctx, int enable) {
    if (!ctx) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        Context& c = ctx->c;
        if (enable && !c.events[0])
            for (cudaEvent_t& e : c.events) BLTC_CUDA(cudaEventCreate(&e));
        c.timing = enable != 0;
        c.marked = 0;
    });
}

bltc_status bltc_last_timings(bltc_context* ctx, float* ms) {
    if (!ctx || !ms) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        Context& c = ctx->c;
        const int pairs[7][2] = {{Context::kStart, Context::kTrees}, {Context::kTrees, Context::kLists},
                                 {Context::kLists, Context::kUpward}, {Context::kUpward, Context::kSweepBegin},
                                 {Context::kSweepBegin, Context::kSweepEnd}, {Context::kSweepEnd, Context::kEnd},
                                 {Context::kStart, Context::kEnd}};
        for (int i = 0; i < 7; ++i) {
            ms[i] = -1.f;
            const unsigned need = (1u << pairs[i][0]) | (1u << pairs[i][1]);
            if ((c.marked & need) != need) continue;
            BLTC_CUDA(cudaEventSynchronize(c.events[pairs[i][1]]));
            BLTC_CUDA(cudaEventElapsedTime(&ms[i], c.events[pairs[i][0]], c.events[pairs[i][1]]));
        }
    });
}

bltc_status bltc_tree_build(bltc_context* ctx, const double* x, const double* y, const double* z,
                            const double* q, int64_t n, int32_t max_leaf, bltc_tree** out) {
    if (!ctx || !out) return BLTC_ERR_ARG;
    *out = nullptr;
    return guarded(ctx, [&] {
        std::unique_ptr<bltc_tree> t(new bltc_tree());
        build_tree(&ctx->c, x, y, z, q, n, max_leaf, &t->t);
        *out = t.release();
    });
}

void bltc_tree_destroy(bltc_tree* tree) {
    if (!tree) return;
    if (tree->t.ctx) cudaSetDevice(tree->t.ctx->device);
    delete tree;
}

bltc_status bltc_tree_info(const bltc_tree* tree, int64_t* n_particles, int64_t* n_nodes,
                           int64_t* n_leaves, int32_t* n_levels) {
    if (!tree) return BLTC_ERR_ARG;
    if (n_particles) *n_particles = tree->t.n;
    if (n_nodes) *n_nodes = tree->t.n_nodes;
    if (n_leaves) *n_leaves = tree->t.n_leaves;
    if (n_levels) *n_levels = tree->t.n_levels;
    return BLTC_OK;
}

bltc_status bltc_tree_export(bltc_context* ctx, const bltc_tree* tree, int64_t* perm, int64_t* begin,
                             int64_t* count, int32_t* parent, int32_t* level, int32_t* n_children,
                             int32_t* children, double* lo, double* hi, double* center, double* radius) {
    if (!ctx || !tree) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        const Tree& t = tree->t;
        Context* c = &ctx->c;
        const int64_t m = t.n_nodes;
        copy_out(c, perm, t.perm.p, t.n);
        copy_out(c, begin, t.begin.p, m);
        copy_out(c, count, t.count.p, m);
        copy_out(c, parent, t.parent.p, m);
        copy_out(c, level, t.level.p, m);
        copy_out(c, n_children, t.nch.p, m);
        copy_out(c, children, t.child.p, 8 * m);
        copy_out(c, lo, t.lo.p, 3 * m);
        copy_out(c, hi, t.hi.p, 3 * m);
        copy_out(c, center, t.center.p, 3 * m);
        copy_out(c, radius, t.radius.p, m);
    });
}

bltc_status bltc_lists_build(bltc_context* ctx, const bltc_tree* batches, const bltc_tree* sources,
                             const bltc_params* params, bltc_lists** out) {
    if (!ctx || !out || !batches || !sources) return BLTC_ERR_ARG;
    *out = nullptr;
    return guarded(ctx, [&] {
        require(params != nullptr, "params is NULL");
        require(params->degree >= 1 && params->degree <= BLTC_MAX_DEGREE, "degree must be in [1, 16]");
        require(std::isfinite(params->theta) && params->theta >= 0.0 && params->theta < 1.0,
                "theta must satisfy 0 <= theta < 1");
        std::unique_ptr<bltc_lists> l(new bltc_lists());
        build_lists(&ctx->c, &batches->t, &sources->t, params->theta, params->degree, &l->l);
        *out = l.release();
    });
}

bltc_status bltc_lists_select(bltc_context* ctx, const bltc_lists* lists, const int32_t* batches,
                              int64_t n_batches, bltc_lists** out) {
    if (!ctx || !lists || !out) return BLTC_ERR_ARG;
    *out = nullptr;
    return guarded(ctx, [&] {
        std::unique_ptr<bltc_lists> l(new bltc_lists());
        select_lists(&ctx->c, &lists->l, batches, n_batches, &l->l);
        *out = l.release();
    });
}

void bltc_lists_destroy(bltc_lists* lists) {
    if (!lists) return;
    if (lists->l.ctx) cudaSetDevice(lists->l.ctx->device);
    delete lists;
}

bltc_status bltc_lists_info(const bltc_lists* lists, int64_t* n_batches, int64_t* n_approx,
                            int64_t* n_direct) {
    if (!lists) return BLTC_ERR_ARG;
    if (n_batches) *n_batches = lists->l.n_batches;
    if (n_approx) *n_approx = lists->l.n_app;
    if (n_direct) *n_direct = lists->l.n_dir;
    return BLTC_OK;
}

bltc_status bltc_lists_export(bltc_context* ctx, const bltc_lists* lists, int64_t* approx_off,
                              int64_t* approx_ids, int64_t* direct_off, int64_t* direct_ids) {
    if (!ctx || !lists) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        const Lists& L = lists->l;
        Context* c = &ctx->c;
        copy_out(c, approx_off, L.app_off.p, L.n_batches + 1);
        copy_out(c, direct_off, L.dir_off.p, L.n_batches + 1);
        copy_out(c, approx_ids, L.app_ids.p, L.n_app);
        copy_out(c, direct_ids, L.dir_ids.p, L.n_dir);
    });
}

bltc_status bltc_stats(bltc_context* ctx, const bltc_lists* lists, int64_t* n_direct_interactions,
                       int64_t* n_approx_interactions) {
    if (!ctx || !lists) return BLTC_ERR_ARG;
    return guarded(ctx, [&] { interaction_counts(&ctx->c, &lists->l, n_direct_interactions, n_approx_interactions); });
}

bltc_status bltc_evaluations(bltc_context* ctx, bltc_lists* lists, const bltc_params* params,
                             int64_t* n_evaluations) {
    if (!ctx || !lists || !n_evaluations) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        check_params(params);
        *n_evaluations = plan_evaluations(&ctx->c, &lists->l, params->degree, params->precision, params->tile);
    });
}

bltc_status bltc_modified_charges(bltc_context* ctx, bltc_tree* sources, const bltc_lists* lists,
                                  const bltc_params* params) {
    if (!ctx || !sources) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        require(params != nullptr, "params is NULL");
        compute_modified_charges(&ctx->c, &sources->t, lists ? &lists->l : nullptr, params->degree,
                                 params->precision);
    });
}

bltc_status bltc_modified_charges_export(bltc_context* ctx, const bltc_tree* sources, double* qhat) {
    if (!ctx || !sources || !qhat) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        const Tree& t = sources->t;
        if (t.q_degree < 1) throw Error(BLTC_ERR_STATE, "no modified charges computed");
        const int64_t np1 = t.q_degree + 1, P = np1 * np1 * np1;
        std::unique_ptr<int32_t[]> slot(new int32_t[t.n_nodes]);
        copy_out(&ctx->c, slot.get(), t.qslot.p, t.n_nodes);
        std::unique_ptr<double[]> q(new double[t.q_slots * P + 1]);
        copy_out(&ctx->c, q.get(), t.qhat64.p, t.q_slots * P);
        for (int64_t v = 0; v < t.n_nodes; ++v)
            for (int64_t k = 0; k < P; ++k)
                qhat[v * P + k] = slot[v] >= 0 ? q[slot[v] * P + k] : std::nan("");
    });
}

bltc_status bltc_evaluate(bltc_context* ctx, const bltc_lists* lists, const bltc_tree* batches,
                          const bltc_tree* sources, const bltc_params* params, double* phi) {
    if (!ctx || !lists || !batches || !sources) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        check_params(params);
        evaluate(&ctx->c, const_cast<Lists*>(&lists->l), &batches->t, &sources->t, *params, phi);
    });
}

bltc_status bltc_solve(bltc_context* ctx, const double* x, const double* y, const double* z,
                       const double* q, int64_t n, const bltc_params* params, double* phi) {
    if (!ctx) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        check_params(params);
        require(x && y && z && q && phi, "solve: NULL pointer");
        solve_device(&ctx->c, x, y, z, q, n, *params, phi);
    });
}

bltc_status bltc_solve_targets(bltc_context* ctx, const double* tx, const double* ty,
                               const double* tz, int64_t nt, const double* sx, const double* sy,
                               const double* sz, const double* sq, int64_t ns,
                               const bltc_params* params, double* phi) {
    if (!ctx) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        check_params(params);
        require(tx && ty && tz && sx && sy && sz && sq && phi, "solve_targets: NULL pointer");
        solve_device_targets(&ctx->c, tx, ty, tz, nt, sx, sy, sz, sq, ns, *params, phi);
    });
}

bltc_status bltc_solve_cp(bltc_context* ctx, const double* tx, const double* ty, const double* tz,
                          int64_t nt, const double* sx, const double* sy, const double* sz,
                          const double* sq, int64_t ns, const bltc_params* params, double* phi) {
    if (!ctx) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        check_params(params);
        require(tx && ty && tz && sx && sy && sz && sq && phi, "solve_cp: NULL pointer");
        solve_device_cp(&ctx->c, tx, ty, tz, nt, sx, sy, sz, sq, ns, *params, phi);
    });
}

bltc_status bltc_solve_cc(bltc_context* ctx, const double* tx, const double* ty, const double* tz,
                          int64_t nt, const double* sx, const double* sy, const double* sz,
                          const double* sq, int64_t ns, const bltc_params* params, double* phi) {
    if (!ctx) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        check_params(params);
        require(tx && ty && tz && sx && sy && sz && sq && phi, "solve_cc: NULL pointer");
        solve_device_cc(&ctx->c, tx, ty, tz, nt, sx, sy, sz, sq, ns, *params, phi);
    });
}

bltc_status bltc_dual_lists(bltc_context* ctx, const bltc_tree* targets, const bltc_tree* sources,
                            const bltc_params* params, int64_t* counts, int64_t* target_ids,
                            int64_t* source_ids) {
    if (!ctx || !targets || !sources || !counts) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        check_params(params);
        DBuf<int2> lists[4];
        int64_t n[4];
        dual_lists(&ctx->c, targets->t, sources->t, params->theta, params->degree, lists, n);
        int64_t o = 0;
        for (int k = 0; k < 4; ++k) {
            counts[k] = n[k];
            if (target_ids && source_ids && n[k] > 0) {
                std::vector<int2> h(static_cast<size_t>(n[k]));
                BLTC_CUDA(cudaMemcpyAsync(h.data(), lists[k].p, sizeof(int2) * n[k], cudaMemcpyDeviceToHost,
                                          ctx->c.stream));
                BLTC_CUDA(cudaStreamSynchronize(ctx->c.stream));
                for (int64_t i = 0; i < n[k]; ++i) {
                    target_ids[o + i] = h[static_cast<size_t>(i)].x;
                    source_ids[o + i] = h[static_cast<size_t>(i)].y;
                }
            }
            o += n[k];
        }
        BLTC_CUDA(cudaStreamSynchronize(ctx->c.stream));
    });
}

bltc_status bltc_solve_hermite(bltc_context* ctx, const double* x, const double* y, const double* z,
                               const double* q, int64_t n, const bltc_params* params, double* phi) {
    if (!ctx) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        check_params(params);
        require(x && y && z && q && phi, "solve_hermite: NULL pointer");
        solve_device_hermite(&ctx->c, x, y, z, q, n, *params, phi);
    });
}

bltc_status bltc_graph_create(bltc_context* ctx, const double* x, const double* y, const double* z,
                              const double* q, int64_t n, const bltc_params* params, double* phi,
                              bltc_graph** out) {
    if (!ctx || !out) return BLTC_ERR_ARG;
    *out = nullptr;
    return guarded(ctx, [&] {
        check_params(params);
        require(x && y && z && q && phi, "graph_create: NULL pointer");
        std::unique_ptr<bltc_graph> h(new bltc_graph());
        h->g = graph_create(&ctx->c, x, y, z, q, n, *params, phi);
        h->ctx = ctx;
        *out = h.release();
    });
}

bltc_status bltc_graph_launch(bltc_context* ctx, bltc_graph* graph) {
    if (!ctx) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        require(graph != nullptr && graph->g != nullptr, "graph_launch: NULL graph");
        if (graph->ctx != ctx) throw Error(BLTC_ERR_STATE, "graph_launch: the graph belongs to another context");
        graph_launch(&ctx->c, graph->g);
    });
}

bltc_status bltc_graph_create_positions(bltc_context* ctx, const double* x, const double* y,
                                        const double* z, const double* q, int64_t n,
                                        const bltc_params* params, double* phi, double headroom,
                                        bltc_graph** out) {
    if (!ctx || !out) return BLTC_ERR_ARG;
    *out = nullptr;
    return guarded(ctx, [&] {
        check_params(params);
        require(x && y && z && q && phi, "graph_create_positions: NULL pointer");
        std::unique_ptr<bltc_graph> h(new bltc_graph());
        h->g = graph_create_positions(&ctx->c, x, y, z, q, n, *params, phi, headroom);
        h->ctx = ctx;
        *out = h.release();
    });
}

bltc_status bltc_graph_info(const bltc_graph* graph, int64_t* out) {
    if (!graph || !graph->g || !out) return BLTC_ERR_ARG;
    graph_info(graph->g, out);
    return BLTC_OK;
}

int64_t bltc_graph_kernels(const bltc_graph* graph) {
    return graph && graph->g ? graph_kernels(graph->g) : -1;
}

void bltc_graph_destroy(bltc_graph* graph) {
    if (!graph) return;
    graph_destroy(graph->g);
    delete graph;
}

bltc_status bltc_solve_host(bltc_context* ctx, const double* x, const double* y, const double* z,
                            const double* q, int64_t n, const bltc_params* params, double* phi) {
    if (!ctx) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        check_params(params);
        require(x && y && z && q && phi, "solve_host: NULL pointer");
        require(n >= 1 && n < (int64_t(1) << 31), "solve_host: n must be in [1, 2^31)");
        Context* c = &ctx->c;
        DBuf<double> dx(c, n), dy(c, n), dz(c, n), dq(c, n), dphi(c, n);
        const size_t bytes = sizeof(double) * n;
        BLTC_CUDA(cudaMemcpyAsync(dx.p, x, bytes, cudaMemcpyHostToDevice, c->stream));
        BLTC_CUDA(cudaMemcpyAsync(dy.p, y, bytes, cudaMemcpyHostToDevice, c->stream));
        BLTC_CUDA(cudaMemcpyAsync(dz.p, z, bytes, cudaMemcpyHostToDevice, c->stream));
        BLTC_CUDA(cudaMemcpyAsync(dq.p, q, bytes, cudaMemcpyHostToDevice, c->stream));
        solve_device(c, dx.p, dy.p, dz.p, dq.p, n, *params, dphi.p);
        BLTC_CUDA(cudaMemcpyAsync(phi, dphi.p, bytes, cudaMemcpyDeviceToHost, c->stream));
        BLTC_CUDA(cudaStreamSynchronize(c->stream));
    });
}

bltc_status bltc_autotune(bltc_context* ctx, const double* x, const double* y, const double* z,
                          const double* q, int64_t n, const bltc_params* params,
                          const int32_t* leaf, const int32_t* batch, int32_t n_candidates,
                          int32_t repeats, int32_t use_cache, bltc_params* best, float* ms) {
    if (!ctx || !best) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        check_params(params);
        require(x && y && z && q, "autotune: NULL pointer");
        require(n >= 1 && n < (int64_t(1) << 31), "autotune: n must be in [1, 2^31)");
        require(leaf && n_candidates >= 1 && repeats >= 1, "autotune: need candidates and repeats");
        for (int i = 0; i < n_candidates; ++i)
            require(leaf[i] >= 1 && (!batch || batch[i] >= 1), "autotune: sizes must be >= 1");
        Context* c = &ctx->c;
        if (ms)
            for (int i = 0; i < n_candidates; ++i) ms[i] = std::nanf("");
        // Screen: the exact work of every candidate from its trees, lists and the sweep's
        // plan (no charges, no sweep).  Candidates whose trees are the same are one candidate.
        struct Cand {
            int64_t s_nodes = 0, b_nodes = 0, b_leaves = 0, cost = 0;
            int same = -1;
        };
        std::vector<Cand> cs(static_cast<size_t>(n_candidates));
        auto screen = [&](int i) {
            bltc_params p = *params;
            p.leaf_size = leaf[i];
            p.batch_size = batch ? batch[i] : leaf[i];
            Tree st;
            build_tree(c, x, y, z, q, n, p.leaf_size, &st);
            std::unique_ptr<Tree> btp;
            const Tree* bt = &st;
            if (p.batch_size != p.leaf_size) {
                btp.reset(new Tree());
                build_tree(c, x, y, z, nullptr, n, p.batch_size, btp.get());
                bt = btp.get();
            }
            Lists L;
            build_lists(c, bt, &st, p.theta, p.degree, &L);
            Cand& k = cs[static_cast<size_t>(i)];
            k.s_nodes = st.n_nodes;
            k.b_nodes = bt->n_nodes;
            k.b_leaves = bt->n_leaves;
            k.cost = plan_slot_cost(c, &L, p.degree, p.precision, p.tile);
            for (int j = 0; j < i; ++j) {
                const Cand& o = cs[static_cast<size_t>(j)];
                if (o.same < 0 && o.s_nodes == k.s_nodes && o.b_nodes == k.b_nodes && o.cost == k.cost) {
                    k.same = j;
                    break;
                }
            }
        };
        screen(0);
        // The distribution enters the cache key as the mean batch size of the first candidate
        // (quarter octaves): a uniform cube and a Plummer sphere of the same size differ there.
        // A cached choice is taken only if it is among this call's candidates.
        int lg = 0;
        while ((int64_t(1) << (lg + 1)) <= n) ++lg;
        const int shape = static_cast<int>(std::lround(4.0 * std::log2(static_cast<double>(n) /
                                                                           static_cast<double>(cs[0].b_leaves))));
        const auto key = std::make_tuple(lg, params->degree, params->kernel, params->precision,
                                         static_cast<int>(std::lround(params->theta * 1000.0)), shape);
        *best = *params;
        if (use_cache) {
            auto it = ctx->tuned.find(key);
            if (it != ctx->tuned.end()) {
                for (int i = 0; i < n_candidates; ++i) {
                    if (leaf[i] == it->second.first && (batch ? batch[i] : leaf[i]) == it->second.second) {
                        best->leaf_size = it->second.first;
                        best->batch_size = it->second.second;
                        return;
                    }
                }
            }
        }
        for (int i = 1; i < n_candidates; ++i) screen(i);
        // Time only the contenders: distinct candidates within kBand of the smallest cost.
        constexpr double kBand = 0.10;
        constexpr int kMaxTimed = 3;
        int64_t min_cost = INT64_MAX;
        for (const Cand& k : cs)
            if (k.same < 0) min_cost = std::min(min_cost, k.cost);
        std::vector<int> cont;
        for (int i = 0; i < n_candidates; ++i) {
            const Cand& k = cs[static_cast<size_t>(i)];
            if (k.same < 0 && static_cast<double>(k.cost) <= (1.0 + kBand) * static_cast<double>(min_cost))
                cont.push_back(i);
        }
        std::stable_sort(cont.begin(), cont.end(), [&](int u, int v) {
            return cs[static_cast<size_t>(u)].cost < cs[static_cast<size_t>(v)].cost;
        });
        if (static_cast<int>(cont.size()) > kMaxTimed) cont.resize(kMaxTimed);
        int win = cont[0];
        if (cont.size() > 1) {
            DBuf<double> phi(c, n);
            cudaEvent_t e0, e1;
            BLTC_CUDA(cudaEventCreate(&e0));
            BLTC_CUDA(cudaEventCreate(&e1));
            float best_ms = 3.0e38f;
            try {
                for (int i : cont) {
                    bltc_params p = *params;
                    p.leaf_size = leaf[i];
                    p.batch_size = batch ? batch[i] : leaf[i];
                    solve_device(c, x, y, z, q, n, p, phi.p);     // warm-up
                    float t_min = 3.0e38f;
                    for (int r = 0; r < repeats; ++r) {
                        BLTC_CUDA(cudaEventRecord(e0, c->stream));
                        solve_device(c, x, y, z, q, n, p, phi.p);
                        BLTC_CUDA(cudaEventRecord(e1, c->stream));
                        BLTC_CUDA(cudaEventSynchronize(e1));
                        float t = 0.f;
                        BLTC_CUDA(cudaEventElapsedTime(&t, e0, e1));
                        t_min = std::min(t_min, t);
                    }
                    if (ms) ms[i] = t_min;
                    if (t_min < best_ms) {
                        best_ms = t_min;
                        win = i;
                    }
                }
            } catch (...) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                throw;
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (ms)
                for (int i = 0; i < n_candidates; ++i)
                    if (cs[static_cast<size_t>(i)].same >= 0) ms[i] = ms[cs[static_cast<size_t>(i)].same];
        }
        best->leaf_size = leaf[win];
        best->batch_size = batch ? batch[win] : leaf[win];
        ctx->tuned[key] = {best->leaf_size, best->batch_size};
    });
}

bltc_status bltc_autotune_tile(bltc_context* ctx, const double* x, const double* y, const double* z,
                               const double* q, int64_t n, const bltc_params* params,
                               const int32_t* tiles, int32_t n_tiles, int32_t repeats,
                               int32_t use_cache, bltc_params* best, float* ms) {
    if (!ctx || !best) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        check_params(params);
        require(x && y && z && q, "autotune_tile: NULL pointer");
        require(n >= 1 && n < (int64_t(1) << 31), "autotune_tile: n must be in [1, 2^31)");
        require(tiles && n_tiles >= 1 && repeats >= 1, "autotune_tile: need candidates and repeats");
        for (int i = 0; i < n_tiles; ++i) require(tile_valid(tiles[i]), "autotune_tile: malformed tile");
        Context* c = &ctx->c;
        if (ms)
            for (int i = 0; i < n_tiles; ++i) ms[i] = std::nanf("");
        // the key of bltc_autotune (the distribution as the mean batch size) plus the sizes
        int64_t n_batches = 0;
        {
            Tree bt;
            build_tree(c, x, y, z, nullptr, n, params->batch_size, &bt);
            n_batches = bt.n_leaves;
        }
        int lg = 0;
        while ((int64_t(1) << (lg + 1)) <= n) ++lg;
        const int shape = static_cast<int>(std::lround(4.0 * std::log2(static_cast<double>(n) /
                                                                           static_cast<double>(n_batches))));
        const auto key = std::make_tuple(lg, params->degree, params->kernel, params->precision,
                                         static_cast<int>(std::lround(params->theta * 1000.0)), shape,
                                         params->leaf_size, params->batch_size);
        *best = *params;
        if (use_cache) {
            auto it = ctx->tuned_tile.find(key);
            if (it != ctx->tuned_tile.end()) {
                for (int i = 0; i < n_tiles; ++i) {
                    if (tiles[i] == it->second) {
                        best->tile = it->second;
                        return;
                    }
                }
            }
        }
        DBuf<double> phi(c, n);
        cudaEvent_t e0, e1;
        BLTC_CUDA(cudaEventCreate(&e0));
        BLTC_CUDA(cudaEventCreate(&e1));
        float best_ms = 3.0e38f;
        int win = 0;
        try {
            for (int i = 0; i < n_tiles; ++i) {
                bltc_params p = *params;
                p.tile = tiles[i];
                solve_device(c, x, y, z, q, n, p, phi.p);     // warm-up
                float t_min = 3.0e38f;
                for (int r = 0; r < repeats; ++r) {
                    BLTC_CUDA(cudaEventRecord(e0, c->stream));
                    solve_device(c, x, y, z, q, n, p, phi.p);
                    BLTC_CUDA(cudaEventRecord(e1, c->stream));
                    BLTC_CUDA(cudaEventSynchronize(e1));
                    float t = 0.f;
                    BLTC_CUDA(cudaEventElapsedTime(&t, e0, e1));
                    t_min = std::min(t_min, t);
                }
                if (ms) ms[i] = t_min;
                if (t_min < best_ms) {
                    best_ms = t_min;
                    win = i;
                }
            }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        best->tile = tiles[win];
        ctx->tuned_tile[key] = tiles[win];
    });
}

bltc_status bltc_kernel_register(bltc_context* ctx, const char* source, int32_t* kernel_id) {
    if (!ctx || !source || !kernel_id) return BLTC_ERR_ARG;
    return guarded(ctx, [&] { *kernel_id = register_user_kernel(&ctx->c, source); });
}

bltc_status bltc_kernel_check(const char* source, int32_t arch, char* log, int64_t len) {
    if (!source) return BLTC_ERR_ARG;
    std::string text;
    bltc_status st = BLTC_OK;
    try {
        if (!compile_user_kernel(source, arch, &text, nullptr)) st = BLTC_ERR_ARG;
    } catch (const Error& e) {
        text = e.what();
        st = e.status;
    } catch (const std::exception& e) {
        text = e.what();
        st = BLTC_ERR_CUDA;
    }
    if (log && len > 0) {
        const int64_t m = std::min<int64_t>(static_cast<int64_t>(text.size()), len - 1);
        std::memcpy(log, text.data(), static_cast<size_t>(m));
        log[m] = '\0';
    }
    return st;
}

bltc_status bltc_direct_sum_noalloc(bltc_context* ctx, const double* tx, const double* ty,
                                    const double* tz, int64_t nt, const double* sx, const double* sy,
                                    const double* sz, const double* sq, int64_t ns,
                                    const bltc_params* params, double* phi) {
    if (!ctx) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        require(params != nullptr, "params is NULL");
        require(params->kernel == BLTC_KERNEL_COULOMB || params->kernel == BLTC_KERNEL_YUKAWA,
                "unknown kernel");
        require(params->kernel != BLTC_KERNEL_YUKAWA || (std::isfinite(params->kappa) && params->kappa >= 0.0),
                "kappa must be finite and >= 0");
        require(params->precision == BLTC_PRECISION_FP64 || params->precision == BLTC_PRECISION_MIXED,
                "unknown precision");
        direct_sum_noalloc(&ctx->c, tx, ty, tz, nt, sx, sy, sz, sq, ns, *params, phi);
    });
}

bltc_status bltc_direct_sum(bltc_context* ctx, const double* tx, const double* ty, const double* tz,
                            int64_t nt, const double* sx, const double* sy, const double* sz,
                            const double* sq, int64_t ns, const bltc_params* params, double* phi) {
    if (!ctx) return BLTC_ERR_ARG;
    return guarded(ctx, [&] {
        require(params != nullptr, "params is NULL");
        require(params->kernel == BLTC_KERNEL_COULOMB || params->kernel == BLTC_KERNEL_YUKAWA,
                "unknown kernel");
        require(params->kernel != BLTC_KERNEL_YUKAWA || (std::isfinite(params->kappa) && params->kappa >= 0.0),
                "kappa must be finite and >= 0");
        require(params->precision == BLTC_PRECISION_FP64 || params->precision == BLTC_PRECISION_MIXED,
                "unknown precision");
        direct_sum(&ctx->c, tx, ty, tz, nt, sx, sy, sz, sq, ns, *params, phi);
    });
}

}  // extern "C"
