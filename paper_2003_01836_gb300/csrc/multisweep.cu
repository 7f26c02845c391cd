// multisweep.cu -- the serving engine's sweeps: work items of several prepared requests in
// slices of persistent launches (MultiSweep, declared in internal.cuh).  Each item runs the
// single-request sweep's device code (sweep_device.cuh) with its own request's arguments, so
// every request's potentials are the bits of bltc_solve of that request alone.
#include <algorithm>
#include <memory>
#include <vector>

#include "internal.cuh"
#include "sweep_device.cuh"

namespace bltc {

using sweepdev::SweepArgs;
// shared with the single-request sweep (sweep.cu)
void check_eval(const Lists* L, const Tree* bt, const Tree* st, const bltc_params& p, const double* phi);
SweepArgs make_args(Context* ctx, const Lists* L, const Tree* bt, const Tree* st, const bltc_params& p,
                    double* partials, unsigned int* counter);
void launch_finalize(Context* ctx, const Lists* L, const Tree* bt, const double* partials,
                     const float* mpart, double* phi);

namespace {

using namespace sweepdev;

// Several requests' sweeps in one persistent launch (the serving engine).  `order` lists
// (request, item) pairs longest first.  The requests' arguments travel in the kernel's
// parameter space (a __grid_constant__ array read through the constant cache), as a single
// request's do.  An item computes exactly what it computes in a single-request launch, so
// every request's potentials are the same bits alone or in a mix.
constexpr int kMultiMax = 64;      // requests per launch: 64 argument sets fit the 32 KB parameter space
struct MultiArgs {
    SweepArgs r[kMultiMax];
};
static_assert(sizeof(MultiArgs) + 64 <= 32764, "the multi-request arguments must fit the kernel parameter space");

template <int KER>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_sweep_multi(const __grid_constant__ MultiArgs m,
                                                             const int2* __restrict__ order,
                                                             int total, unsigned int* counter) {
    extern __shared__ __align__(16) float4 sm_dyn[];
    float4* sm = sm_dyn;
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(counter, 1u));
        __syncthreads();
        const int i = s_item;
        if (i >= total) return;
        const int2 o = order[i];
        const SweepArgs& a = m.r[o.x];
        item_mixed<KER>(a, a.items[o.y], sm);
    }
}

}  // namespace

struct MultiSweep::Job {
    SweepJob j;
    void* tag = nullptr;
    uint64_t seq = 0;
    DBuf<double> partials;
    DBuf<float> mpart;
    int64_t next = 0;                 // first item (in the plan's longest-first order) not run
    int64_t remaining = 0;            // weighted cost of the items not run
};

// Pinned host and device staging of one slice's item order, reused once its event completed.
struct MultiSweep::Slot {
    int2* host = nullptr;
    int64_t cap = 0;
    DBuf<int2> dev;
    DBuf<unsigned int> counters;
    cudaEvent_t start = nullptr, done = nullptr;   // around the launch group, timed
    bool used = false;
    int64_t cost = 0, budget = 0;                   // its weighted work and the slice's budget
    bool measured = true;
};

MultiSweep::MultiSweep(Context* ctx) : ctx_(ctx) {
    for (int i = 0; i < 2; ++i) {
        slots_.emplace_back(new Slot());
        BLTC_CUDA(cudaEventCreate(&slots_.back()->start));
        BLTC_CUDA(cudaEventCreate(&slots_.back()->done));
    }
}

MultiSweep::~MultiSweep() {
    for (auto& sl : slots_) {
        if (sl->done) {
            cudaEventSynchronize(sl->done);
            cudaEventDestroy(sl->done);
        }
        if (sl->start) cudaEventDestroy(sl->start);
        if (sl->host) cudaFreeHost(sl->host);
    }
}

// A Yukawa evaluation costs about 1.5 times a Coulomb one (one MUFU.EX2 beside the RSQ).
static int64_t weighted_cost(int64_t cost, const bltc_params& p) {
    return p.kernel == BLTC_KERNEL_YUKAWA ? cost + cost / 2 : cost;
}

void MultiSweep::add(const SweepJob& job, void* tag) {
    require(job.p.precision == BLTC_PRECISION_MIXED, "serving runs the mixed-precision sweep");
    check_eval(job.L, job.bt, job.st, job.p, job.phi);
    if (!job.L->plan.valid || job.L->plan.degree != job.p.degree || job.L->plan.tile != job.p.tile ||
        job.L->plan.mutual != (job.L->bt == job.L->st && job.L->n_dir > 0))
        throw Error(BLTC_ERR_STATE, "multi sweep: request has no work plan");
    const Plan& pl = job.L->plan;
    std::unique_ptr<Job> jb(new Job());
    jb->j = job;
    jb->tag = tag;
    jb->seq = seq_++;
    jb->partials = DBuf<double>(ctx_, pl.partial_len);
    jb->mpart = DBuf<float>(ctx_, pl.mutual ? pl.mpart_len : 0);
    for (int64_t c : pl.h_cost) jb->remaining += weighted_cost(c, job.p);
    jobs_.push_back(std::move(jb));
}

// After a launch group has run: its weighted work over its device time updates the engine's
// rate (an exponential average over the groups that filled at least half of their slice's
// budget, so that short tails do not count as slow work).
void MultiSweep::measure(Slot& sl) {
    if (!sl.used || sl.measured) return;
    sl.measured = true;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, sl.start, sl.done) != cudaSuccess || ms <= 0.f) {
        cudaGetLastError();
        return;
    }
    if (sl.budget > 0 && 2 * sl.cost < sl.budget) return;
    const double r = static_cast<double>(sl.cost) / (1e3 * static_cast<double>(ms));
    rate_ = rate_ > 0.0 ? 0.7 * rate_ + 0.3 * r : r;
}

void MultiSweep::wait_in_flight(int keep) {
    // slots alternate: next_slot_ is the older one, next_slot_ ^ 1 the most recent
    Slot& older = *slots_[static_cast<size_t>(next_slot_)];
    if (older.used) {
        BLTC_CUDA(cudaEventSynchronize(older.done));
        measure(older);
    }
    if (keep == 0) {
        Slot& recent = *slots_[static_cast<size_t>(next_slot_ ^ 1)];
        if (recent.used) {
            BLTC_CUDA(cudaEventSynchronize(recent.done));
            measure(recent);
        }
    }
}

std::vector<void*> MultiSweep::tags() const {
    std::vector<void*> t;
    for (const auto& jb : jobs_) t.push_back(jb->tag);
    return t;
}

void MultiSweep::clear() {
    cudaStreamSynchronize(ctx_->stream);
    jobs_.clear();
}

int MultiSweep::run_slice(int64_t budget, int max_requests, std::vector<void*>* finished) {
    if (jobs_.empty()) return 0;
    cudaStream_t s = ctx_->stream;
    // the requests with the least remaining work first (arrival order on ties)
    std::vector<Job*> byrem;
    for (auto& jb : jobs_) byrem.push_back(jb.get());
    std::stable_sort(byrem.begin(), byrem.end(), [](const Job* x, const Job* y) {
        return x->remaining != y->remaining ? x->remaining < y->remaining : x->seq < y->seq;
    });
    // items of this slice: (job, first item, end item), whole requests first, the last one in part
    struct Take {
        Job* jb;
        int64_t i0, i1;
    };
    std::vector<Take> take;
    int64_t got = 0;
    for (Job* jb : byrem) {
        if (static_cast<int>(take.size()) >= std::max(1, max_requests)) break;
        if (budget > 0 && got >= budget) break;
        const Plan& pl = jb->j.L->plan;
        int64_t i = jb->next;
        while (i < pl.n_items && (budget <= 0 || got < budget)) {
            const int64_t c = weighted_cost(pl.h_cost[static_cast<size_t>(i)], jb->j.p);
            got += c;
            jb->remaining -= c;
            ++i;
        }
        if (i > jb->next) take.push_back(Take{jb, jb->next, i});
        jb->next = i;
    }
    const int64_t cap = std::max<int64_t>(
        1, kMinBlocks * static_cast<int64_t>(std::max(1, ctx_->sm_count)) - free_blocks_);
    BLTC_CUDA(cudaFuncSetAttribute(k_sweep_multi<BLTC_KERNEL_COULOMB>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmem));
    BLTC_CUDA(cudaFuncSetAttribute(k_sweep_multi<BLTC_KERNEL_YUKAWA>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmem));
    for (size_t t0 = 0; t0 < take.size(); t0 += kMultiMax) {
        const size_t t1 = std::min(take.size(), t0 + kMultiMax);
        std::unique_ptr<MultiArgs> m(new MultiArgs());
        std::vector<std::pair<int64_t, int2>> all;
        for (size_t t = t0; t < t1; ++t) {
            Job* jb = take[t].jb;
            const Plan& pl = jb->j.L->plan;
            SweepArgs& sa = m->r[t - t0];
            sa = make_args(ctx_, jb->j.L, jb->j.bt, jb->j.st, jb->j.p, jb->partials.p, nullptr);
            sa.mpart = pl.mutual ? jb->mpart.p : nullptr;
            for (int64_t i = take[t].i0; i < take[t].i1; ++i)
                all.push_back({pl.h_cost[static_cast<size_t>(i)], make_int2(static_cast<int>(t - t0), static_cast<int>(i))});
        }
        // longest first within the launch, one persistent launch per kernel type present
        std::stable_sort(all.begin(), all.end(), [](const std::pair<int64_t, int2>& x,
                                                    const std::pair<int64_t, int2>& y) { return x.first > y.first; });
        Slot& sl = *slots_[static_cast<size_t>(next_slot_)];
        next_slot_ ^= 1;
        if (sl.used) {
            BLTC_CUDA(cudaEventSynchronize(sl.done));     // its previous slice has run
            measure(sl);
        }
        sl.cost = 0;
        for (const auto& pr : all) sl.cost += weighted_cost(pr.first, take[t0 + pr.second.x].jb->j.p);
        sl.budget = budget;
        sl.measured = false;
        const int64_t total = static_cast<int64_t>(all.size());
        if (total > sl.cap) {
            if (sl.host) cudaFreeHost(sl.host);
            sl.host = nullptr;
            sl.cap = std::max<int64_t>(total, 2 * sl.cap);
            BLTC_CUDA(cudaMallocHost(&sl.host, sizeof(int2) * sl.cap));
        }
        if (!sl.dev.p || sl.dev.n < total) sl.dev = DBuf<int2>(ctx_, sl.cap);
        if (!sl.counters.p) sl.counters = DBuf<unsigned int>(ctx_, 2);
        int64_t nc = 0;
        for (const auto& pr : all)
            if (take[t0 + pr.second.x].jb->j.p.kernel != BLTC_KERNEL_YUKAWA) sl.host[nc++] = pr.second;
        int64_t ny = nc;
        for (const auto& pr : all)
            if (take[t0 + pr.second.x].jb->j.p.kernel == BLTC_KERNEL_YUKAWA) sl.host[ny++] = pr.second;
        BLTC_CUDA(cudaEventRecord(sl.start, s));
        BLTC_CUDA(cudaMemsetAsync(sl.counters.p, 0, 2 * sizeof(unsigned int), s));
        BLTC_CUDA(cudaMemcpyAsync(sl.dev.p, sl.host, sizeof(int2) * total, cudaMemcpyHostToDevice, s));
        if (nc > 0) {
            k_sweep_multi<BLTC_KERNEL_COULOMB><<<static_cast<unsigned>(std::min<int64_t>(nc, cap)), kThreads, kMixedSmem, s>>>(
                *m, sl.dev.p, static_cast<int>(nc), sl.counters.p); ++ctx_->launches;
            BLTC_LAUNCH_CHECK("sweep multi coulomb");
        }
        if (total > nc) {
            k_sweep_multi<BLTC_KERNEL_YUKAWA><<<static_cast<unsigned>(std::min<int64_t>(total - nc, cap)), kThreads, kMixedSmem, s>>>(
                *m, sl.dev.p + nc, static_cast<int>(total - nc), sl.counters.p + 1); ++ctx_->launches;
            BLTC_LAUNCH_CHECK("sweep multi yukawa");
        }
        BLTC_CUDA(cudaEventRecord(sl.done, s));
        sl.used = true;
    }
    // finalize the requests whose items have all run; their buffers are freed in stream order
    for (size_t k = 0; k < jobs_.size();) {
        Job* jb = jobs_[k].get();
        const Plan& pl = jb->j.L->plan;
        if (jb->next < pl.n_items) {
            ++k;
            continue;
        }
        launch_finalize(ctx_, jb->j.L, jb->j.bt, jb->partials.p, jb->mpart.p, jb->j.phi);
        finished->push_back(jb->tag);
        jobs_.erase(jobs_.begin() + static_cast<std::ptrdiff_t>(k));
    }
    if (jobs_.empty()) {
        // idle: the device staging goes back to the allocator (freed after its last use in
        // stream order); the pinned host staging stays for the next request
        for (auto& sl : slots_) {
            sl->dev.reset();
            sl->counters.reset();
        }
    }
    return static_cast<int>(take.size());
}

}  // namespace bltc
