// internal.cuh -- data structures and helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "bltc.h"

namespace bltc {

// Failure inside the library; converted to a bltc_status at the C boundary.
struct Error : std::runtime_error {
    bltc_status status;
    Error(bltc_status s, const std::string& m) : std::runtime_error(m), status(s) {}
};

#define BLTC_CUDA(call)                                                                   \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            throw ::bltc::Error(BLTC_ERR_CUDA, std::string(#call) + ": " +                \
                                                   cudaGetErrorString(e_));               \
    } while (0)

#define BLTC_LAUNCH_CHECK(what)                                                           \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess)                                                            \
            throw ::bltc::Error(BLTC_ERR_CUDA, std::string("launch ") + (what) + ": " +   \
                                                   cudaGetErrorString(e_));               \
    } while (0)

inline void require(bool ok, const std::string& msg) {
    if (!ok) throw Error(BLTC_ERR_ARG, msg);
}

struct Context {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;
    bltc_alloc_fn alloc_fn = nullptr;
    bltc_free_fn free_fn = nullptr;
    void* alloc_user = nullptr;
    std::string err;
    double* cheb_t[BLTC_MAX_DEGREE + 1] = {};   // device: t_k = cos(pi k / n), k = 0..n
    int64_t* pinned = nullptr;                  // small pinned host buffer for counters
    static constexpr int kPinnedWords = 64;
    int64_t launches = 0;                       // kernels launched through this context
    bool capturing = false;                     // inside a graph capture: no allocation allowed
    // A second stream for work that overlaps the host-synchronising setup of the main stream
    // (created on first use): fork() makes it wait for the main stream's work so far, join()
    // makes the main stream wait for it.
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    void fork();
    void join();
    uint64_t next_serial = 1;
    // Optional phase timing: CUDA events recorded on the stream at the phase boundaries.
    enum Mark { kStart, kTrees, kLists, kUpward, kSweepBegin, kSweepEnd, kEnd, kMarks };
    bool timing = false;
    cudaEvent_t events[kMarks] = {};
    unsigned marked = 0;
    void mark(Mark m) {
        if (!timing) return;
        if (m == kStart) marked = 0;
        if (m == kSweepBegin) marked &= ~((1u << kSweepBegin) | (1u << kSweepEnd) | (1u << kEnd));
        if (cudaEventRecord(events[m], stream) == cudaSuccess) marked |= 1u << m;
    }

    // A bump arena that serves every allocation while it is set (the capture of a solve sized
    // on the device, which allocates nothing while captured): blocks are never freed one by
    // one, the arena's owner frees it whole.  With `measure` set, allocations are served as
    // usual and their arena footprint is summed in `measured`.
    struct Arena {
        char* base = nullptr;
        size_t size = 0, used = 0;
        bool measure = false;
        size_t measured = 0;
        static size_t footprint(size_t bytes) { return (bytes + 255) & ~static_cast<size_t>(255); }
    };
    Arena arena;
    bool in_arena() const { return arena.base != nullptr; }
    void* dalloc(size_t bytes);
    void dfree(void* p, size_t bytes);
    // Every allocation is rounded up to 16 bytes so small counters can be read as words.
    template <typename T>
    static size_t bytes_for(int64_t count) {
        size_t b = sizeof(T) * static_cast<size_t>(count > 0 ? count : 1);
        return (b + 15) & ~static_cast<size_t>(15);
    }
    template <typename T>
    T* alloc(int64_t count) {
        return static_cast<T*>(dalloc(bytes_for<T>(count)));
    }
    // Copies `words` int64 values from device to the pinned buffer and waits.
    const int64_t* read_words(const void* dev, int words);
    const double* cheb_table(int degree);
    // User kernels (bltc_kernel_register): run-time compiled sweeps, id USER_BASE + index.
    struct UserKernel {
        cudaLibrary_t lib = nullptr;
        cudaKernel_t mixed = nullptr, fp64 = nullptr;
    };
    std::vector<UserKernel> user_kernels;
    const UserKernel& user_kernel(int id) const {
        const int i = id - BLTC_KERNEL_USER_BASE;
        if (i < 0 || i >= static_cast<int>(user_kernels.size()))
            throw Error(BLTC_ERR_ARG, "kernel id is not a kernel registered in this context");
        return user_kernels[static_cast<size_t>(i)];
    }
};

// RAII device buffer from the context allocator.
template <typename T>
struct DBuf {
    Context* ctx = nullptr;
    T* p = nullptr;
    int64_t n = 0;
    DBuf() = default;
    // memory from the context's arena is not freed by the buffer (ctx stays null)
    DBuf(Context* c, int64_t count) : ctx(c->in_arena() ? nullptr : c), p(c->alloc<T>(count)), n(count) {}
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : ctx(o.ctx), p(o.p), n(o.n) { o.p = nullptr; }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) {
            reset();
            ctx = o.ctx;
            p = o.p;
            n = o.n;
            o.p = nullptr;
        }
        return *this;
    }
    ~DBuf() { reset(); }
    void reset() {
        if (p && ctx) ctx->dfree(p, Context::bytes_for<T>(n));
        p = nullptr;
    }
    T* release() {
        T* q = p;
        p = nullptr;
        return q;
    }
};

// Capacities of a setup sized on the device (a solve for new positions captured as one CUDA
// graph).  The host-driven setup reads each count back before it allocates and launches the
// next step.  Sized on the device, every buffer is allocated once at its capacity, every count
// stays in device memory, kernels launch over the capacity and skip what lies beyond the
// count, and a solve that would exceed a capacity raises `flag` (device memory, 0 = all held)
// instead of writing past it.  Entries beyond a count are inert: nodes with level -1, no
// particles and no children; batches with leaf id -1; list counts of 0.
struct Caps {
    int32_t nodes = 0;                // tree nodes
    int32_t levels = 0;               // level iterations of the tree build
    int32_t level_nodes = 0;          // nodes of one level
    int64_t chunks = 0;               // particle chunks of one level
    int64_t app = 0, dir = 0;         // list entries
    int32_t slots = 0;                // clusters with modified charges
    int32_t up_items = 0;             // leaf-sum items of the upward pass
    int32_t m2m = 0;                  // marked internal nodes of one level
    int64_t items = 0;                // sweep work items
    int64_t partial_len = 0;          // item partials (doubles)
    int64_t mpart_len = 0;            // mutual rows (floats)
    int32_t* flag = nullptr;          // device overflow flag
};

// A built tree (nodes in DFS pre-order; particles in tree order).
struct Tree {
    Context* ctx = nullptr;
    int64_t n = 0;
    int32_t max_leaf = 0;
    int64_t n_nodes = 0, n_leaves = 0;  // sized on the device: the capacities
    int32_t n_levels = 0;
    bool has_q = false;
    const Caps* caps = nullptr;       // non-null: sized on the device
    DBuf<int32_t> dcount;             // sized on the device: {nodes, leaves} in device memory
    DBuf<double> px, py, pz, pq;      // particles in tree order
    DBuf<int32_t> perm;               // perm[i] = original index
    DBuf<int32_t> begin, count, parent, level, nch, child;  // child: 8 per node
    DBuf<double> lo, hi, center, radius;                    // lo/hi/center: 3 per node
    DBuf<int32_t> leaves;             // leaf node ids in DFS order
    // modified charges for one (degree, precision)
    int q_degree = -1, q_precision = -1;
    uint64_t q_lists = 0;             // serial of the lists the charges were computed for (0: all)
    int64_t q_slots = 0;
    DBuf<int32_t> qslot;              // per node: row of qhat, or -1
    DBuf<double> qhat64;              // [q_slots * P]
    DBuf<float> qhat32;               // [q_slots * P] (mixed precision)
};

// Per-batch work items of one evaluation (cached in the lists).
struct Plan {
    bool valid = false;
    int degree = -1;
    int tile = 0;                     // bltc_params.tile the plan was built for
    bool mutual = false;              // mutual leaf pairs evaluated once (mixed, batches = sources)
    int64_t mpart_len = 0;            // doubles of mutual rows
    DBuf<int64_t> dir_moff;           // per direct entry: its mutual row in mpart, or -1
    int64_t n_items = 0;
    int64_t partial_len = 0;
    DBuf<int4> items;                 // {batch, e0, e1, chunk}
    DBuf<int64_t> part_off;           // per batch: first partial
    DBuf<int32_t> n_chunks;           // per batch
    DBuf<uint8_t> dir_sel;            // per direct entry: bit 0 self-pair test, bit 1 close-pair
                                      // check, bit 2 mutual owner, bit 3 mutual partner (skip)
    DBuf<float> dir_tau2;             // per direct entry: r^2 below which pairs are redone in FP64
    std::vector<int64_t> h_cost;      // host copy of the items' interaction counts (queue order)
    // sized on the device: the plan's totals ({cost, items, partial length, mutual length}) and
    // the sweep's first item (the sorted items fill the end of the capacity)
    DBuf<int64_t> dwords;
    DBuf<int32_t> dstart;
};

struct Lists {
    Context* ctx = nullptr;
    uint64_t serial = 0;              // unique per context, never 0
    const Tree* bt = nullptr;
    const Tree* st = nullptr;
    double theta = 0.0;
    int degree = 0;
    int64_t n_batches = 0, n_app = 0, n_dir = 0;   // sized on the device: the capacities
    DBuf<int32_t> app_off, app_ids, dir_off, dir_ids;
    const Caps* caps = nullptr;       // non-null: sized on the device
    DBuf<int32_t> dcount;             // sized on the device: {approximation, direct} entries
    Plan plan;
};

// ---- steps (implemented in tree.cu, lists.cu, upward.cu, sweep.cu, direct.cu) -------
void build_tree(Context* ctx, const double* x, const double* y, const double* z,
                const double* q, int64_t n, int32_t max_leaf, Tree* out,
                const Caps* caps = nullptr);
void build_lists(Context* ctx, const Tree* bt, const Tree* st, double theta, int degree,
                 Lists* out, const Caps* caps = nullptr);
// The lists of the selected batches only (strictly increasing batch indices); the other
// batches get empty lists.
void select_lists(Context* ctx, const Lists* L, const int32_t* sel, int64_t n_sel, Lists* out);
void compute_modified_charges(Context* ctx, Tree* st, const Lists* lists, int degree,
                              int precision);
// The upward pass in two parts: prepare_upward marks the clusters, allocates the modified
// charges in the tree and the pass's work lists (host synchronisation); run_upward only
// launches kernels (no allocation, no synchronisation), so it can be captured in a graph.
struct UpwardPlan {
    int degree = 0, precision = 0;
    const Caps* caps = nullptr;      // non-null: sized on the device (counts below are capacities)
    DBuf<int32_t> dcount;            // {slots, items} in device memory
    DBuf<int32_t> lev;               // sized on the device: per level count, offset, cursor
    int32_t n_slots = 0, n_items = 0, chunk = 1;
    DBuf<int32_t> slot_node, item0, list;
    DBuf<int4> items;
    DBuf<double> partial, scratch;
    std::vector<int32_t> h, off;     // marked internal nodes per level and their offsets in list
};
void prepare_upward(Context* ctx, Tree* st, const Lists* lists, int degree, int precision,
                    UpwardPlan* up);
void run_upward(Context* ctx, Tree* st, const UpwardPlan& up);

// The whole of Algorithm 1 (api.cu): trees, lists, upward pass beside the plan, sweep.
void solve_device(Context* c, const double* x, const double* y, const double* z,
                  const double* q, int64_t n, const bltc_params& p, double* phi);
// Capacities of a tree from its node arrays (tree.cu): nodes, levels, the widest level, the
// most particle chunks of a level.  Reads the tree back to the host.
void tree_counts(Context* ctx, const Tree& t, Caps* caps);

// A solve captured as one CUDA graph (graph.cu): with fixed positions (only the charges are
// read at a launch) or, sized on the device, for new positions at every launch.
struct GraphSolve;
GraphSolve* graph_create(Context* c, const double* x, const double* y, const double* z, const double* q,
                         int64_t n, const bltc_params& p, double* phi);
GraphSolve* graph_create_positions(Context* c, const double* x, const double* y, const double* z,
                                   const double* q, int64_t n, const bltc_params& p, double* phi,
                                   double headroom);
// {kernels per launch, launches, launches redone on the host path, captures}
void graph_info(const GraphSolve* g, int64_t out[4]);
void graph_launch(Context* c, GraphSolve* g);
int64_t graph_kernels(const GraphSolve* g);
void graph_destroy(GraphSolve* g);
void evaluate(Context* ctx, Lists* lists, const Tree* bt, const Tree* st,
              const bltc_params& p, double* phi);
// evaluate in parts: the work plan (prepare_plan), the sweep's scratch, and the launches
// alone (run_sweep: no allocation, no synchronisation), for capture in a graph.
struct SweepBuffers {
    DBuf<double> partials;
    DBuf<float> mpart;
    DBuf<unsigned int> counter;
};
void alloc_sweep_buffers(Context* ctx, const Lists* lists, SweepBuffers* b);
void run_sweep(Context* ctx, Lists* lists, const Tree* bt, const Tree* st, const bltc_params& p,
               double* phi, const SweepBuffers& b);
void interaction_counts(Context* ctx, const Lists* lists, int64_t* n_dir, int64_t* n_app);
// Work plan of a list set (items, partial layout, self-pair flags); built once per degree.
void build_plan(Context* ctx, Lists* L, int degree, bool mutual, int tile = 0);
// The plan for an evaluation in `precision` (mutual pairs for MIXED with batches = sources)
// with the sweep's tile shape `tile` (bltc_params.tile).
void prepare_plan(Context* ctx, Lists* L, int degree, int precision, int tile = 0);
// Kernel evaluations the sweep performs for that plan (mutual pairs counted once).
int64_t plan_evaluations(Context* ctx, Lists* L, int degree, int precision, int tile = 0);
// The sweep's cost model for that plan: evaluations with every batch padded to the target
// slots its source groups run (the autotuner's screen).
int64_t plan_slot_cost(Context* ctx, Lists* L, int degree, int precision, int tile = 0);
// The fields of bltc_params.tile (0: the defaults).
inline int tile_group_cap(int tile) { return (tile & 15) ? (tile & 15) : 8; }
inline int tile_items_per_block(int tile) { return ((tile >> 4) & 255) ? ((tile >> 4) & 255) : 16; }
inline bool tile_valid(int tile) {
    const int g = tile & 15;
    return (tile >> 12) == 0 && (g == 0 || g == 1 || g == 2 || g == 4 || g == 8);
}
// The Hermite treecode's sweep (sweep.cu) and the whole solve (hermite.cu).
void evaluate_hermite(Context* ctx, Lists* L, const Tree* bt, const Tree* st, const bltc_params& p,
                      const double* qh64, const float* qh32, const int32_t* qslot, double* phi);
void solve_device_hermite(Context* c, const double* x, const double* y, const double* z, const double* q,
                          int64_t n, const bltc_params& p, double* phi);
// The cluster-particle variant (cp.cu): targets interpolated, sources summed exactly.
void solve_device_cp(Context* c, const double* tx, const double* ty, const double* tz, int64_t nt,
                     const double* sx, const double* sy, const double* sz, const double* sq, int64_t ns,
                     const bltc_params& p, double* phi);
// The cluster-cluster variant (cp.cu): dual tree traversal, then the same sweeps.
void solve_device_cc(Context* c, const double* tx, const double* ty, const double* tz, int64_t nt,
                     const double* sx, const double* sy, const double* sz, const double* sq, int64_t ns,
                     const bltc_params& p, double* phi);
// The dual traversal's CC, CP, PC and PP lists as (target node, source node) pairs.
void dual_lists(Context* c, const Tree& tt, const Tree& st, double theta, int degree,
                DBuf<int2> (&lists)[4], int64_t (&counts)[4]);
// Compiles the sweeps for a user kernel given as CUDA source (user_kernel.cu); returns its id.
int register_user_kernel(Context* ctx, const char* source);
// Compiles a user kernel's sweeps for sm_<arch> without a device and returns the compiler
// log; true when it compiled.
bool compile_user_kernel(const char* source, int arch, std::string* log, std::vector<char>* cubin);
// One request of a multi-request sweep: its lists, trees, parameters and device phi.
struct SweepJob {
    Lists* L;
    const Tree* bt;
    const Tree* st;
    bltc_params p;
    double* phi;
};
// Mixed-precision sweeps of several prepared requests, in slices (the serving engine).  A
// request is added when it is ready; run_slice launches work items worth about `budget`
// interactions (all of them when budget <= 0), taken from the requests with the least
// remaining work first, at most max_requests of them, as persistent launches of at most 64
// requests each, then the finalize of every request whose items have all run, and returns
// those requests' tags.  An item computes the same bits in any launch, so every request's
// potentials equal evaluate() of that request alone.
class MultiSweep {
public:
    explicit MultiSweep(Context* ctx);
    ~MultiSweep();
    MultiSweep(const MultiSweep&) = delete;
    MultiSweep& operator=(const MultiSweep&) = delete;
    void add(const SweepJob& job, void* tag);      // checks the job, allocates its partials
    // block slots the persistent launches leave free (for other streams' kernels)
    void set_free_blocks(int n) { free_blocks_ = n > 0 ? n : 0; }
    // waits until at most `keep` (0 or 1) enqueued launch groups may still be running
    void wait_in_flight(int keep);
    // weighted interactions per microsecond the launches have run at (0 before any measure)
    double rate() const { return rate_; }
    bool idle() const { return jobs_.empty(); }
    std::vector<void*> tags() const;                // requests with work still to run
    void clear();                                   // drops every request (after a failure)
    // returns the number of requests the slice took items from
    int run_slice(int64_t budget, int max_requests, std::vector<void*>* finished);

private:
    struct Job;
    struct Slot;
    Context* ctx_;
    std::vector<std::unique_ptr<Job>> jobs_;
    std::vector<std::unique_ptr<Slot>> slots_;      // staging of the item order, two in flight
    int next_slot_ = 0;
    uint64_t seq_ = 0;
    int free_blocks_ = 0;
    double rate_ = 0.0;
    void measure(Slot& sl);
};
void direct_sum(Context* ctx, const double* tx, const double* ty, const double* tz,
                int64_t nt, const double* sx, const double* sy, const double* sz,
                const double* sq, int64_t ns, const bltc_params& p, double* phi);

// bltc_direct_sum without any allocation: partial sums in a fixed file-scope device array.
void direct_sum_noalloc(Context* ctx, const double* tx, const double* ty, const double* tz,
                        int64_t nt, const double* sx, const double* sy, const double* sz,
                        const double* sq, int64_t ns, const bltc_params& p, double* phi);

// ---- device-wide exclusive scan (scan.cu) -------------------------------------------
// out[i] = sum_{j<i} in[i]; *total (device, may be null) = sum of all.
void exclusive_scan_i32(Context* ctx, const int32_t* in, int32_t* out, int64_t n,
                        int32_t* total);
void exclusive_scan_i64(Context* ctx, const int64_t* in, int64_t* out, int64_t n,
                        int64_t* total);

// 32-byte aligned (x, y, z, q) record for FP64 shared-memory staging.
struct __align__(32) D4 {
    double x, y, z, w;
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline unsigned grid_for(int64_t n, int threads, int64_t cap = 1 << 20) {
    int64_t g = ceil_div(n, threads);
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return static_cast<unsigned>(g);
}

}  // namespace bltc
