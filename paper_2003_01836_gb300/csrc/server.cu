// server.cu -- the serving runtime: continuous batching of treecode requests on one GPU.
//
// Requests (particle systems of any size, each with its own parameters) are queued by
// bltc_server_submit and admitted in arrival order while their estimated device memory fits
// the HBM budget.  Admitted requests are prepared by setup workers -- host threads, each with
// its own stream -- which copy the inputs in and build the tree, the interaction lists, the
// modified charges and the work plan (steps A0-A2 and the plan).  The sweep engine thread
// takes every request that is ready and runs the far- and near-field sweeps of the requests
// in its hands in slices: each slice takes the work items worth about slice_us microseconds
// from the requests with the least remaining work first (at most max_batch requests), runs
// them as persistent launches (items longest first), then finalizes every request whose
// items have all run.  A request that becomes ready while a large one is being swept joins
// at the next slice instead of waiting for the whole large sweep; slice_us = 0 runs all the
// ready work in one slice.  A completer thread waits for the finalize, copies each potential
// back to the caller's buffer, frees the request's device memory and returns its budget.
// While slices run, the workers prepare the next requests on their own streams, so setup and
// sweeps of different requests overlap on the device.
//
// A request's work items depend only on the request, and an item computes the same bits in
// any launch, so every potential equals bltc_solve of that request alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "internal.cuh"

namespace bltc {

static double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Device bytes a request may hold at its peak, per particle and fixed: inputs 32 B, tree copy
// 36 B, build buffers 73 B, potentials 8 B, work-item partials (at most ~24 items per batch
// at 8 B per target), plus nodes, lists and modified charges.
static int64_t estimate_bytes(int64_t n, const bltc_params& p) {
    const int64_t np1 = p.degree + 1, P = np1 * np1 * np1;
    const int64_t leaves = n / std::max(1, std::min(p.leaf_size, p.batch_size)) + 1;
    const int64_t nodes = 4 * leaves + 64;
    return 400 * n + nodes * (256 + 12 * P + 64) + leaves * 4096 + (32 << 20);
}

struct ServerRequest {
    uint64_t ticket = 0;
    const double *hx = nullptr, *hy = nullptr, *hz = nullptr, *hq = nullptr;
    double* hphi = nullptr;
    int64_t n = 0;
    bltc_params p{};
    enum State { kQueued, kAdmitted, kReady, kDone } state = kQueued;
    bltc_status status = BLTC_OK;
    std::string err;
    int64_t bytes = 0;
    double t_submit = 0, t_admit = 0, t_ready = 0, t_done = 0, t_swept = 0, t_copy = 0;
    int batch = 0;
    // device state, allocated through the preparing worker's context
    std::vector<DBuf<double>> X;
    DBuf<double> phi;
    std::unique_ptr<Tree> st, bt;
    std::unique_ptr<Lists> L;
    cudaEvent_t ready_ev = nullptr;
};

struct Server {
    bltc_server_config cfg{};
    int64_t budget = 0;
    cudaMemPool_t pool = nullptr;
    std::vector<std::unique_ptr<Context>> worker_ctx;
    std::unique_ptr<Context> engine_ctx, completer_ctx;
    std::mutex mu;
    std::condition_variable cv;     // any state change
    std::deque<ServerRequest*> queued, ready;
    std::deque<std::pair<std::vector<ServerRequest*>, cudaEvent_t>> inflight;
    std::unordered_map<uint64_t, std::unique_ptr<ServerRequest>> reqs;
    int64_t in_use = 0, peak_in_use = 0;
    std::atomic<int64_t> live{0}, peak_live{0};
    uint64_t next_ticket = 1;
    int64_t n_submitted = 0, n_completed = 0, n_failed = 0, n_cancelled = 0, n_launches = 0;
    int64_t max_batch_seen = 0;
    bool engine_failed = false;      // the engine could not start: requests fail at submission
    int64_t preparing = 0;          // admitted, not yet ready or failed
    std::string last_err;           // message of the most recent failed request
    bool stop = false;
    std::vector<std::thread> threads;
};

// The server's contexts allocate from one shared pool and account the live bytes.
static void* server_alloc(size_t bytes, void* stream, void* user) {
    Server* s = static_cast<Server*>(user);
    void* p = nullptr;
    if (cudaMallocFromPoolAsync(&p, bytes, s->pool, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const int64_t v = s->live.fetch_add(static_cast<int64_t>(bytes)) + static_cast<int64_t>(bytes);
    int64_t pk = s->peak_live.load();
    while (v > pk && !s->peak_live.compare_exchange_weak(pk, v)) {
    }
    return p;
}

static void server_free(void* ptr, size_t bytes, void* stream, void* user) {
    Server* s = static_cast<Server*>(user);
    cudaFreeAsync(ptr, static_cast<cudaStream_t>(stream));
    s->live.fetch_sub(static_cast<int64_t>(bytes));
}

// A context on its own stream: the setup workers' streams take the greatest priority, so
// their kernels get the block slots the sweeps leave free, and free slots between slices,
// before the next slice's blocks.
static std::unique_ptr<Context> make_context(Server* s, bool urgent) {
    std::unique_ptr<Context> c(new Context());
    c->device = s->cfg.device;
    BLTC_CUDA(cudaSetDevice(c->device));
    BLTC_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
    int least = 0, greatest = 0;
    BLTC_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    BLTC_CUDA(cudaStreamCreateWithPriority(&c->stream, cudaStreamNonBlocking, urgent ? greatest : least));
    BLTC_CUDA(cudaMallocHost(&c->pinned, sizeof(int64_t) * Context::kPinnedWords));
    c->alloc_fn = server_alloc;
    c->free_fn = server_free;
    c->alloc_user = s;
    return c;
}

static void release_context(Context* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) {
        cudaStreamSynchronize(c->stream);
        cudaStreamDestroy(c->stream);
    }
    for (double*& t : c->cheb_t)
        if (t) cudaFree(t);
    if (c->pinned) cudaFreeHost(c->pinned);
}

// Frees a request's device memory (its last use has completed).
static void drop_device_state(ServerRequest* r) {
    r->L.reset();
    r->bt.reset();
    r->st.reset();
    r->phi.reset();
    r->X.clear();
    if (r->ready_ev) {
        cudaEventDestroy(r->ready_ev);
        r->ready_ev = nullptr;
    }
}

static void finish(Server* s, ServerRequest* r, bltc_status st, const std::string& err) {
    // caller holds s->mu
    r->status = st;
    r->err = err;
    if (st != BLTC_OK && st != BLTC_ERR_CANCELLED) s->last_err = err;
    r->state = ServerRequest::kDone;
    r->t_done = now_s();
    s->in_use -= r->bytes;
    if (st == BLTC_OK)
        ++s->n_completed;
    else if (st == BLTC_ERR_CANCELLED)
        ++s->n_cancelled;
    else
        ++s->n_failed;
    s->cv.notify_all();
}

// Steps A0-A2 and the work plan of one request, on the worker's stream.
static void prepare(Context* c, ServerRequest* r) {
    const int64_t n = r->n;
    const size_t bytes = sizeof(double) * static_cast<size_t>(n);
    const double* h[4] = {r->hx, r->hy, r->hz, r->hq};
    for (int k = 0; k < 4; ++k) {
        r->X.emplace_back(c, n);
        BLTC_CUDA(cudaMemcpyAsync(r->X.back().p, h[k], bytes, cudaMemcpyHostToDevice, c->stream));
    }
    r->phi = DBuf<double>(c, n);
    r->st.reset(new Tree());
    build_tree(c, r->X[0].p, r->X[1].p, r->X[2].p, r->X[3].p, n, r->p.leaf_size, r->st.get());
    const Tree* bt = r->st.get();
    if (r->p.batch_size != r->p.leaf_size) {
        r->bt.reset(new Tree());
        build_tree(c, r->X[0].p, r->X[1].p, r->X[2].p, nullptr, n, r->p.batch_size, r->bt.get());
        bt = r->bt.get();
    }
    r->L.reset(new Lists());
    build_lists(c, bt, r->st.get(), r->p.theta, r->p.degree, r->L.get());
    compute_modified_charges(c, r->st.get(), r->L.get(), r->p.degree, r->p.precision);
    prepare_plan(c, r->L.get(), r->p.degree, r->p.precision, r->p.tile);
    BLTC_CUDA(cudaEventCreateWithFlags(&r->ready_ev, cudaEventDisableTiming));
    BLTC_CUDA(cudaEventRecord(r->ready_ev, c->stream));
}

static void worker_loop(Server* s, Context* c) {
    cudaSetDevice(s->cfg.device);
    for (;;) {
        ServerRequest* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                return s->stop ||
                       (!s->queued.empty() && s->in_use + s->queued.front()->bytes <= s->budget);
            });
            if (s->stop) return;
            r = s->queued.front();
            s->queued.pop_front();
            r->state = ServerRequest::kAdmitted;
            r->t_admit = now_s();
            s->in_use += r->bytes;
            s->peak_in_use = std::max(s->peak_in_use, s->in_use);
            ++s->preparing;
        }
        std::string err;
        bltc_status st = BLTC_OK;
        try {
            prepare(c, r);
        } catch (const Error& e) {
            st = e.status;
            err = e.what();
        } catch (const std::exception& e) {
            st = BLTC_ERR_CUDA;
            err = e.what();
        }
        if (st != BLTC_OK) {
            cudaStreamSynchronize(c->stream);
            drop_device_state(r);
            std::lock_guard<std::mutex> lk(s->mu);
            --s->preparing;
            finish(s, r, st, err);
            s->cv.notify_all();
            continue;
        }
        std::lock_guard<std::mutex> lk(s->mu);
        --s->preparing;
        r->state = ServerRequest::kReady;
        r->t_ready = now_s();
        s->ready.push_back(r);
        s->cv.notify_all();
    }
}

// Weighted interactions the sweep runs per microsecond, about (1e6 cube, Coulomb): converts the
// slice duration asked for into a work budget until the engine has measured its own rate.
constexpr double kInteractionsPerUs = 3.5e6;

static void engine_loop(Server* s) {
    Context* c = s->engine_ctx.get();
    cudaSetDevice(s->cfg.device);
    std::unique_ptr<MultiSweep> ms;
    try {
        ms.reset(new MultiSweep(c));
        ms->set_free_blocks(s->cfg.setup_blocks);
    } catch (const std::exception& e) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->last_err = e.what();
        s->engine_failed = true;
        s->cv.notify_all();
        return;
    }
    for (;;) {
        std::vector<ServerRequest*> add;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->ready.empty() || !ms->idle(); });
            if (s->stop && s->ready.empty() && ms->idle()) return;
            if (ms->idle() && s->cfg.linger_us > 0) {
                // batching window: wait for requests still in preparation (or queued)
                const auto until = std::chrono::steady_clock::now() +
                                   std::chrono::microseconds(s->cfg.linger_us);
                s->cv.wait_until(lk, until, [&] {
                    return s->stop || static_cast<int>(s->ready.size()) >= s->cfg.max_batch ||
                           (s->preparing == 0 && s->queued.empty());
                });
            }
        }
        // At most slices_in_flight - 1 earlier slices stay enqueued; the requests that became
        // ready meanwhile join the slice assembled next.
        try {
            ms->wait_in_flight(s->cfg.slices_in_flight == 2 ? 1 : 0);
        } catch (const std::exception&) {
            // a failed slice is reported by the launch that follows
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            while (!s->ready.empty()) {
                add.push_back(s->ready.front());
                s->ready.pop_front();
            }
        }
        std::vector<void*> fin;
        int took = 0;
        bltc_status st = BLTC_OK;
        std::string err;
        try {
            for (ServerRequest* r : add) {
                BLTC_CUDA(cudaStreamWaitEvent(c->stream, r->ready_ev, 0));
                ms->add(SweepJob{r->L.get(), r->bt ? r->bt.get() : r->st.get(), r->st.get(), r->p, r->phi.p}, r);
            }
            // the slice's work from the rate its launches have run at (the request mix's cost per
            // interaction varies with theta, the degree and the kernel)
            const double rate = ms->rate() > 0.0 ? ms->rate() : kInteractionsPerUs;
            const int64_t budget = s->cfg.slice_us > 0 ? static_cast<int64_t>(rate * s->cfg.slice_us) : 0;
            took = ms->run_slice(budget, s->cfg.max_batch, &fin);
        } catch (const Error& e) {
            st = e.status;
            err = e.what();
        } catch (const std::exception& e) {
            st = BLTC_ERR_CUDA;
            err = e.what();
        }
        if (st != BLTC_OK) {
            // every request with work in the engine fails
            std::vector<void*> tags = ms->tags();
            for (ServerRequest* r : add)
                if (std::find(tags.begin(), tags.end(), static_cast<void*>(r)) == tags.end() &&
                    std::find(fin.begin(), fin.end(), static_cast<void*>(r)) == fin.end())
                    tags.push_back(r);
            for (void* t : fin) tags.push_back(t);
            ms->clear();
            std::lock_guard<std::mutex> lk(s->mu);
            ++s->n_launches;
            for (void* t : tags) {
                ServerRequest* r = static_cast<ServerRequest*>(t);
                drop_device_state(r);
                finish(s, r, st, err);
            }
            continue;
        }
        cudaEvent_t done = nullptr;
        if (!fin.empty()) {
            if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventRecord(done, c->stream) != cudaSuccess) {
                cudaStreamSynchronize(c->stream);
                if (done) cudaEventDestroy(done);
                done = nullptr;
            }
        }
        std::lock_guard<std::mutex> lk(s->mu);
        ++s->n_launches;
        s->max_batch_seen = std::max<int64_t>(s->max_batch_seen, static_cast<int64_t>(took));
        if (!fin.empty()) {
            std::vector<ServerRequest*> batch;
            const double t = now_s();
            for (void* f : fin) {
                ServerRequest* r = static_cast<ServerRequest*>(f);
                r->batch = took;
                r->t_swept = t;
                batch.push_back(r);
            }
            s->inflight.emplace_back(std::move(batch), done);
            s->cv.notify_all();
        }
    }
}

static void completer_loop(Server* s) {
    Context* c = s->completer_ctx.get();
    cudaSetDevice(s->cfg.device);
    for (;;) {
        std::pair<std::vector<ServerRequest*>, cudaEvent_t> job;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->inflight.empty(); });
            if (s->inflight.empty()) {
                if (s->stop) return;
                continue;
            }
            job = std::move(s->inflight.front());
            s->inflight.pop_front();
        }
        if (job.second) {
            cudaEventSynchronize(job.second);
            cudaEventDestroy(job.second);
        }
        const double t_copy = now_s();
        for (ServerRequest* r : job.first) {
            r->t_copy = t_copy;
            cudaError_t e = cudaMemcpyAsync(r->hphi, r->phi.p, sizeof(double) * static_cast<size_t>(r->n),
                                            cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            drop_device_state(r);
            std::lock_guard<std::mutex> lk(s->mu);
            finish(s, r, e == cudaSuccess ? BLTC_OK : BLTC_ERR_CUDA,
                   e == cudaSuccess ? "" : std::string("copy-out: ") + cudaGetErrorString(e));
        }
    }
}

}  // namespace bltc

using namespace bltc;

struct bltc_server {
    Server s;
};

extern "C" {

bltc_status bltc_server_create(const bltc_server_config* cfg, bltc_server** out) {
    if (!cfg || !out) return BLTC_ERR_ARG;
    *out = nullptr;
    if (cfg->setup_workers < 1 || cfg->setup_workers > 64 || cfg->max_batch < 1 || cfg->hbm_budget_bytes < 0 ||
        cfg->linger_us < 0 || cfg->slice_us < 0 || cfg->setup_blocks < 0 || cfg->slices_in_flight < 0 ||
        cfg->slices_in_flight > 2)
        return BLTC_ERR_ARG;
    std::unique_ptr<bltc_server> h(new bltc_server());
    Server& s = h->s;
    s.cfg = *cfg;
    try {
        int ndev = 0;
        BLTC_CUDA(cudaGetDeviceCount(&ndev));
        if (cfg->device < 0 || cfg->device >= ndev) return BLTC_ERR_ARG;
        BLTC_CUDA(cudaSetDevice(cfg->device));
        size_t free_b = 0, total_b = 0;
        BLTC_CUDA(cudaMemGetInfo(&free_b, &total_b));
        s.budget = cfg->hbm_budget_bytes > 0 ? cfg->hbm_budget_bytes : static_cast<int64_t>(0.8 * free_b);
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = cfg->device;
        BLTC_CUDA(cudaMemPoolCreate(&s.pool, &props));
        uint64_t keep = ~0ULL;
        cudaMemPoolSetAttribute(s.pool, cudaMemPoolAttrReleaseThreshold, &keep);
        const bool urgent = cfg->setup_blocks > 0;
        for (int w = 0; w < cfg->setup_workers; ++w) s.worker_ctx.push_back(make_context(&s, urgent));
        s.engine_ctx = make_context(&s, false);
        s.completer_ctx = make_context(&s, urgent);
    } catch (const Error& e) {
        for (auto& c : s.worker_ctx) release_context(c.get());
        release_context(s.engine_ctx.get());
        release_context(s.completer_ctx.get());
        if (s.pool) cudaMemPoolDestroy(s.pool);
        return e.status;
    }
    for (auto& c : s.worker_ctx) s.threads.emplace_back(worker_loop, &s, c.get());
    s.threads.emplace_back(engine_loop, &s);
    s.threads.emplace_back(completer_loop, &s);
    *out = h.release();
    return BLTC_OK;
}

bltc_status bltc_server_submit(bltc_server* h, const double* x, const double* y, const double* z,
                               const double* q, int64_t n, const bltc_params* p, double* phi,
                               uint64_t* ticket) {
    if (!h || !x || !y || !z || !q || !phi || !p || !ticket) return BLTC_ERR_ARG;
    if (n < 1 || n >= (int64_t(1) << 31)) return BLTC_ERR_ARG;
    if (p->degree < 1 || p->degree > BLTC_MAX_DEGREE || !(p->theta >= 0.0 && p->theta < 1.0) ||
        p->leaf_size < 1 || p->batch_size < 1 || !tile_valid(p->tile) ||
        (p->kernel != BLTC_KERNEL_COULOMB && p->kernel != BLTC_KERNEL_YUKAWA) ||
        (p->kernel == BLTC_KERNEL_YUKAWA && !(p->kappa >= 0.0 && p->kappa < 1e300)) ||
        p->precision != BLTC_PRECISION_MIXED)
        return BLTC_ERR_ARG;
    Server& s = h->s;
    std::unique_ptr<ServerRequest> r(new ServerRequest());
    r->hx = x;
    r->hy = y;
    r->hz = z;
    r->hq = q;
    r->hphi = phi;
    r->n = n;
    r->p = *p;
    r->bytes = estimate_bytes(n, *p);
    r->t_submit = now_s();
    std::lock_guard<std::mutex> lk(s.mu);
    if (s.stop || s.engine_failed) return BLTC_ERR_STATE;
    if (r->bytes > s.budget) return BLTC_ERR_OOM;
    r->ticket = s.next_ticket++;
    *ticket = r->ticket;
    s.queued.push_back(r.get());
    s.reqs.emplace(r->ticket, std::move(r));
    ++s.n_submitted;
    s.cv.notify_all();
    return BLTC_OK;
}

bltc_status bltc_server_wait(bltc_server* h, uint64_t ticket, double timeout_s, bltc_request_info* info) {
    if (!h) return BLTC_ERR_ARG;
    Server& s = h->s;
    std::unique_lock<std::mutex> lk(s.mu);
    auto it = s.reqs.find(ticket);
    if (it == s.reqs.end()) return BLTC_ERR_ARG;
    ServerRequest* r = it->second.get();
    auto done = [&] { return r->state == ServerRequest::kDone; };
    if (timeout_s < 0) {
        s.cv.wait(lk, done);
    } else if (!s.cv.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
        return BLTC_ERR_TIMEOUT;
    }
    if (info) {
        info->status = r->status;
        info->batch = r->batch;
        info->bytes_reserved = r->bytes;
        info->t_submit = r->t_submit;
        info->t_admit = r->t_admit;
        info->t_ready = r->t_ready;
        info->t_done = r->t_done;
        info->t_swept = r->t_swept;
        info->t_copy = r->t_copy;
    }
    const bltc_status st = r->status;
    s.reqs.erase(it);
    return st;
}

bltc_status bltc_server_cancel(bltc_server* h, uint64_t ticket) {
    if (!h) return BLTC_ERR_ARG;
    Server& s = h->s;
    std::lock_guard<std::mutex> lk(s.mu);
    auto it = s.reqs.find(ticket);
    if (it == s.reqs.end()) return BLTC_ERR_ARG;
    ServerRequest* r = it->second.get();
    if (r->state != ServerRequest::kQueued) return BLTC_ERR_STATE;
    s.queued.erase(std::find(s.queued.begin(), s.queued.end(), r));
    r->bytes = 0;
    finish(&s, r, BLTC_ERR_CANCELLED, "cancelled");
    return BLTC_OK;
}

bltc_status bltc_server_stats(bltc_server* h, bltc_server_counters* out) {
    if (!h || !out) return BLTC_ERR_ARG;
    Server& s = h->s;
    std::lock_guard<std::mutex> lk(s.mu);
    out->submitted = s.n_submitted;
    out->completed = s.n_completed;
    out->failed = s.n_failed;
    out->cancelled = s.n_cancelled;
    out->queued = static_cast<int64_t>(s.queued.size());
    out->sweep_launches = s.n_launches;
    out->max_batch = s.max_batch_seen;
    out->budget_bytes = s.budget;
    out->reserved_bytes = s.in_use;
    out->peak_reserved_bytes = s.peak_in_use;
    out->live_bytes = s.live.load();
    out->peak_live_bytes = s.peak_live.load();
    return BLTC_OK;
}

int64_t bltc_server_last_error(bltc_server* h, char* buf, int64_t len) {
    if (!h) return -1;
    Server& s = h->s;
    std::lock_guard<std::mutex> lk(s.mu);
    const int64_t n = static_cast<int64_t>(s.last_err.size());
    if (buf && len > 0) {
        const int64_t m = std::min<int64_t>(n, len - 1);
        std::memcpy(buf, s.last_err.data(), static_cast<size_t>(m));
        buf[m] = '\0';
    }
    return n;
}

void bltc_server_destroy(bltc_server* h) {
    if (!h) return;
    Server& s = h->s;
    {
        // cancel what was not admitted; admitted requests run to completion
        std::lock_guard<std::mutex> lk(s.mu);
        for (ServerRequest* r : s.queued) {
            r->bytes = 0;
            finish(&s, r, BLTC_ERR_CANCELLED, "cancelled");
        }
        s.queued.clear();
    }
    {
        std::unique_lock<std::mutex> lk(s.mu);
        s.cv.wait(lk, [&] {
            for (auto& kv : s.reqs)
                if (kv.second->state != ServerRequest::kDone) return false;
            return true;
        });
        s.stop = true;
        s.cv.notify_all();
    }
    for (std::thread& t : s.threads) t.join();
    for (auto& kv : s.reqs) drop_device_state(kv.second.get());
    for (auto& c : s.worker_ctx) release_context(c.get());
    release_context(s.engine_ctx.get());
    release_context(s.completer_ctx.get());
    if (s.pool) cudaMemPoolDestroy(s.pool);
    delete h;
}

}  // extern "C"
