// sweep.cu -- A3/A4/A5: far-field and near-field batch-cluster sums and the finalize.
//
// Far field (Eq. 11): phi_i += sum_k G(x_i, s_k) qhat_k over the (n+1)^3 Chebyshev points
// s_k = (s1[k1], s2[k2], s3[k3]) of each approximated cluster.  Near field (Eq. 9):
// phi_i += sum_{y_j in C} G(x_i, y_j) q_j over each directly summed cluster.
//
// GB300 mapping.  The target batch is the unit of work, as in the paper (the MAC is applied
// per batch so all its targets share one list, Sec. III-B "Target Batching").  Each
// batch's combined list (approximated clusters, then direct clusters) is cut into items of
// roughly equal interaction count; one persistent launch of (SMs x 2) blocks pulls items
// from an atomic counter.  A block holds up to 256*T targets in registers (T per thread),
// stages one cluster at a time in shared memory (sources as float4 (x, y, z, q) relative
// to the batch centre, or the proxy grid: 3 x (n+1) point coordinates and (n+1)^3
// modified charges), and every thread streams the staged sources against its T targets.
// The proxy grid is used in tensor form: for each (k1, k2) the partial r^2 of a target is
// reused across the n+1 values of k3 (Eq. 8's tensor product).  Each item writes one
// partial potential per target; the finalize sums a target's partials in item order (FP64)
// and scatters to the caller's order, so results are deterministic (the paper used atomics
// across four streams instead, Sec. III-B "Asynchronous Streams").
//
// Precision.  MIXED: kernel evaluations in FP32 on coordinates taken relative to the batch
// centre (the FP64 differences rounded once), FP32 sums over one staged tile, FP64 across
// tiles and clusters.  FP64: every operation in double on absolute coordinates.
// A pair with r^2 == 0 (a target meeting itself) is skipped; for the far field theta < 1
// keeps every proxy point away from every target, so no test is needed there.
#include <algorithm>
#include <memory>
#include <vector>

#include "internal.cuh"
#include "sweep_device.cuh"

namespace bltc {
namespace {

using namespace sweepdev;

template <int KER>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_sweep_mixed(SweepArgs a) {
    sweep_mixed_body<KER>(a);
}

template <int KER>
__global__ void __launch_bounds__(kThreads, 2) k_sweep_fp64(SweepArgs a) {
    sweep_fp64_body<KER>(a);
}

template <int KER>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_sweep_hermite_mixed(SweepArgs a) {
    sweep_mixed_body<KER, true>(a);
}

template <int KER>
__global__ void __launch_bounds__(kThreads, 2) k_sweep_hermite(SweepArgs a) {
    sweep_hermite_body<KER>(a);
}

// Adds rows [r, n) of s_row, read as T, to this thread's U targets; kAhead rows are loaded
// before they are added, so every thread keeps several independent loads in flight.
template <typename T, int U, int kAhead>
__device__ __forceinline__ void add_rows(const void* const* s_row, int r, int n, int t0, int nb,
                                         double (&s)[U]) {
    for (; r + kAhead <= n; r += kAhead) {
        double v[kAhead][U];
#pragma unroll
        for (int k = 0; k < kAhead; ++k) {
            const T* row = static_cast<const T*>(s_row[r + k]);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0 + static_cast<int>(threadIdx.x) + u * static_cast<int>(blockDim.x);
                v[k][u] = t < nb ? static_cast<double>(row[t]) : 0.0;
            }
        }
#pragma unroll
        for (int k = 0; k < kAhead; ++k)
#pragma unroll
            for (int u = 0; u < U; ++u) s[u] += v[k][u];
    }
    for (; r < n; ++r) {
        const T* row = static_cast<const T*>(s_row[r]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + static_cast<int>(threadIdx.x) + u * static_cast<int>(blockDim.x);
            if (t < nb) s[u] += static_cast<double>(row[t]);
        }
    }
}

// Per target: its items' partials (FP64) in item order, then (mutual pairs) the FP32 rows that
// partner batches wrote for it, in list order; scattered to the caller's order.  Each thread
// keeps 8 targets so that every row is read with 8 independent, coalesced loads in flight.
__global__ void k_finalize(const int32_t* __restrict__ b_leaves, const int32_t* __restrict__ b_begin,
                           const int32_t* __restrict__ b_count, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ n_chunks, const int64_t* __restrict__ part_off,
                           const double* __restrict__ partials, const int32_t* __restrict__ dir_off,
                           const uint8_t* __restrict__ dir_sel, const int64_t* __restrict__ dir_moff,
                           const float* __restrict__ mpart, double* __restrict__ phi,
                           const int32_t* __restrict__ stop) {
    constexpr int U = 8;          // targets per thread
    constexpr int kRows = 256;    // row pointers gathered per round
    constexpr int kAhead = 4;     // rows loaded before they are added
    __shared__ const void* s_row[kRows];
    __shared__ int s_n, s_nd;
    __shared__ bool s_more;
    const int b = blockIdx.x;
    const int B = b_leaves[b];
    // sized on the device: no batch here, or a capacity was exceeded (the solve is redone)
    if (B < 0 || (stop && *stop)) return;
    const int tb = b_begin[B], nb = b_count[B], K = n_chunks[b];
    const double* p = partials + part_off[b];
    const int e1 = dir_off[b + 1];
    const int lane = static_cast<int>(threadIdx.x) & 31;
    for (int t0 = 0; t0 < nb; t0 += U * static_cast<int>(blockDim.x)) {
        double s[U];
#pragma unroll
        for (int u = 0; u < U; ++u) s[u] = 0.0;
        // The rows are added in a fixed order: the item partials, then (mutual pairs) the partner
        // rows of the skipped entries in list order.  Warp 0 gathers their addresses in rounds
        // (its own progress in r0 and e), the item rows of a round first; every thread then adds
        // the round's rows.
        int r0 = 0, e = dir_off[b];
        for (;;) {
            __syncthreads();
            if (threadIdx.x < 32) {
                int n = 0;
                for (; r0 < K && n < kRows; ++r0, ++n)
                    if (lane == 0) s_row[n] = p + static_cast<int64_t>(r0) * nb;
                const int nd = n;
                if (mpart && r0 >= K) {
                    while (e < e1 && n <= kRows - 32) {
                        const int ee = e + lane;
                        const bool skip = ee < e1 && (dir_sel[ee] & kSelSkip);
                        const unsigned v = __ballot_sync(0xffffffffu, skip);
                        if (skip) s_row[n + __popc(v & ((1u << lane) - 1u))] = mpart + dir_moff[ee];
                        n += __popc(v);
                        e += 32;
                    }
                }
                if (lane == 0) {
                    s_n = n;
                    s_nd = nd;
                    s_more = r0 < K || (mpart != nullptr && e < e1);
                }
            }
            __syncthreads();
            const int n = s_n, nd = s_nd;
            const bool more = s_more;
            add_rows<double, U, kAhead>(s_row, 0, nd, t0, nb, s);
            add_rows<float, U, kAhead>(s_row, nd, n, t0, nb, s);
            if (!more) break;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + static_cast<int>(threadIdx.x) + u * static_cast<int>(blockDim.x);
            if (t < nb) phi[perm[tb + t]] = s[u];
        }
    }
}

// The persistent sweep's queue counter: the first real item, or the capacity when the setup
// exceeded a capacity (the sweep then runs nothing and the solve is redone on the host path).
__global__ void k_counter_start(unsigned int* counter, const int32_t* __restrict__ start,
                                const int32_t* __restrict__ stop, int64_t cap) {
    *counter = *stop ? static_cast<unsigned int>(cap) : static_cast<unsigned int>(*start);
}

}  // namespace

void check_eval(const Lists* L, const Tree* bt, const Tree* st, const bltc_params& p,
                const double* phi) {
    if (L->bt != bt || L->st != st)
        throw Error(BLTC_ERR_STATE, "evaluate: lists were built for other trees");
    if (L->degree != p.degree)
        throw Error(BLTC_ERR_STATE, "evaluate: lists were built for another degree");
    if (st->q_degree != p.degree || st->q_precision != p.precision)
        throw Error(BLTC_ERR_STATE, "evaluate: modified charges missing for this degree/precision");
    if (!st->has_q) throw Error(BLTC_ERR_STATE, "evaluate: source tree has no charges");
    if (st->q_lists != 0 && st->q_lists != L->serial)
        throw Error(BLTC_ERR_STATE, "evaluate: modified charges were computed for other lists");
    require(phi != nullptr, "evaluate: phi is NULL");
}

SweepArgs make_args(Context* ctx, const Lists* L, const Tree* bt, const Tree* st,
                    const bltc_params& p, double* partials, unsigned int* counter) {
    const Plan& pl = L->plan;
    SweepArgs a{};
    a.b_leaves = bt->leaves.p;
    a.b_begin = bt->begin.p;
    a.b_count = bt->count.p;
    a.b_center = bt->center.p;
    a.b_lo = bt->lo.p;
    a.b_hi = bt->hi.p;
    a.tx = bt->px.p;
    a.ty = bt->py.p;
    a.tz = bt->pz.p;
    a.s_begin = st->begin.p;
    a.s_count = st->count.p;
    a.s_lo = st->lo.p;
    a.s_hi = st->hi.p;
    a.sx = st->px.p;
    a.sy = st->py.p;
    a.sz = st->pz.p;
    a.sq = st->pq.p;
    a.qslot = st->qslot.p;
    a.qhat64 = st->qhat64.p;
    a.qhat32 = st->qhat32.p;
    a.cheb_t = ctx->cheb_table(p.degree);
    a.np1 = p.degree + 1;
    a.app_off = L->app_off.p;
    a.app_ids = L->app_ids.p;
    a.dir_off = L->dir_off.p;
    a.dir_ids = L->dir_ids.p;
    a.dir_sel = pl.dir_sel.p;
    a.dir_tau2 = pl.dir_tau2.p;
    a.dir_moff = pl.mutual ? pl.dir_moff.p : nullptr;
    a.mpart = nullptr;
    a.items = pl.items.p;
    a.part_off = pl.part_off.p;
    a.partials = partials;
    a.n_items = static_cast<int>(pl.n_items);
    a.counter = counter;
    a.kernel = p.kernel;
    const double kappa = p.kernel == BLTC_KERNEL_COULOMB ? 0.0 : p.kappa;
    a.kappa = kappa;
    a.neg_kappa_log2e = static_cast<float>(-kappa * 1.4426950408889634);
    a.param32 = static_cast<float>(kappa);
    a.g_max = tile_group_cap(p.tile);
    return a;
}


void evaluate(Context* ctx, Lists* L, const Tree* bt, const Tree* st, const bltc_params& p,
              double* phi) {
    check_eval(L, bt, st, p, phi);
    prepare_plan(ctx, L, p.degree, p.precision, p.tile);
    SweepBuffers b;
    alloc_sweep_buffers(ctx, L, &b);
    run_sweep(ctx, L, bt, st, p, phi, b);
}

void alloc_sweep_buffers(Context* ctx, const Lists* L, SweepBuffers* b) {
    const Plan& pl = L->plan;
    b->partials = DBuf<double>(ctx, pl.partial_len);
    b->mpart = DBuf<float>(ctx, pl.mutual ? pl.mpart_len : 0);
    b->counter = DBuf<unsigned int>(ctx, 1);
}

void run_sweep(Context* ctx, Lists* L, const Tree* bt, const Tree* st, const bltc_params& p,
               double* phi, const SweepBuffers& b) {
    cudaStream_t s = ctx->stream;
    const Plan& pl = L->plan;
    if (L->caps) {
        k_counter_start<<<1, 1, 0, s>>>(b.counter.p, pl.dstart.p, L->caps->flag, pl.n_items); ++ctx->launches;
    } else {
        BLTC_CUDA(cudaMemsetAsync(b.counter.p, 0, sizeof(unsigned int), s));
    }
    SweepArgs a = make_args(ctx, L, bt, st, p, b.partials.p, b.counter.p);
    a.mpart = pl.mutual ? b.mpart.p : nullptr;
    const int per_sm = p.precision == BLTC_PRECISION_MIXED ? kMinBlocks : 2;
    const unsigned grid = static_cast<unsigned>(
        std::min<int64_t>(pl.n_items, per_sm * static_cast<int64_t>(std::max(1, ctx->sm_count))));
    ctx->mark(Context::kSweepBegin);
    if (pl.n_items > 0 && p.kernel >= BLTC_KERNEL_USER_BASE) {
        // a registered user kernel: the same sweeps, compiled at run time with its G
        const Context::UserKernel& uk = ctx->user_kernel(p.kernel);
        void* args[] = {const_cast<SweepArgs*>(&a)};
        const bool mixed = p.precision == BLTC_PRECISION_MIXED;
        BLTC_CUDA(cudaLaunchKernel(reinterpret_cast<const void*>(mixed ? uk.mixed : uk.fp64), dim3(grid),
                                   dim3(kThreads), args, mixed ? kMixedSmem : 0, s)); ++ctx->launches;
        BLTC_LAUNCH_CHECK("sweep (user kernel)");
    } else if (pl.n_items > 0) {
        if (p.precision == BLTC_PRECISION_MIXED) {
            if (p.kernel == BLTC_KERNEL_YUKAWA) {
                BLTC_CUDA(cudaFuncSetAttribute(k_sweep_mixed<BLTC_KERNEL_YUKAWA>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmem));
                k_sweep_mixed<BLTC_KERNEL_YUKAWA><<<grid, kThreads, kMixedSmem, s>>>(a); ++ctx->launches;
            } else {
                BLTC_CUDA(cudaFuncSetAttribute(k_sweep_mixed<BLTC_KERNEL_COULOMB>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmem));
                k_sweep_mixed<BLTC_KERNEL_COULOMB><<<grid, kThreads, kMixedSmem, s>>>(a); ++ctx->launches;
            }
        } else {
            if (p.kernel == BLTC_KERNEL_YUKAWA) {
                k_sweep_fp64<BLTC_KERNEL_YUKAWA><<<grid, kThreads, 0, s>>>(a); ++ctx->launches;
            } else {
                k_sweep_fp64<BLTC_KERNEL_COULOMB><<<grid, kThreads, 0, s>>>(a); ++ctx->launches;
            }
        }
        BLTC_LAUNCH_CHECK("sweep");
    }
    ctx->mark(Context::kSweepEnd);
    k_finalize<<<static_cast<unsigned>(L->n_batches), 256, 0, s>>>(
        bt->leaves.p, bt->begin.p, bt->count.p, bt->perm.p, pl.n_chunks.p, pl.part_off.p,
        b.partials.p, L->dir_off.p, pl.dir_sel.p, a.dir_moff, a.mpart, phi,
        L->caps ? L->caps->flag : nullptr); ++ctx->launches;
    BLTC_LAUNCH_CHECK("finalize");
    ctx->mark(Context::kEnd);
}

// The Hermite treecode's sweep: Hermite far field with charges [slot][8][(n+1)^3] (qh64 for
// FP64, qh32 for mixed precision), the treecode's near field, then the finalize.  The lists
// were built with degree 2n+1, whose (2n+2)^3 = 8 (n+1)^3 points give the Hermite size test
// and the cost of an approximation.
void evaluate_hermite(Context* ctx, Lists* L, const Tree* bt, const Tree* st, const bltc_params& p,
                      const double* qh64, const float* qh32, const int32_t* qslot, double* phi) {
    cudaStream_t s = ctx->stream;
    require(L->bt == bt && L->st == st, "hermite: lists were built for other trees");
    require(L->degree == 2 * p.degree + 1, "hermite: lists were built for another degree");
    const bool mixed = p.precision == BLTC_PRECISION_MIXED;
    prepare_plan(ctx, L, L->degree, p.precision, p.tile);
    Plan& pl = L->plan;
    DBuf<double> partials(ctx, pl.partial_len);
    DBuf<float> mpart(ctx, pl.mutual ? pl.mpart_len : 0);
    DBuf<unsigned int> counter(ctx, 1);
    BLTC_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned int), s));
    SweepArgs a = make_args(ctx, L, bt, st, p, partials.p, counter.p);
    a.np1 = p.degree + 1;
    a.qhat64 = qh64;
    a.qhat32 = qh32;
    a.qslot = qslot;
    a.mpart = pl.mutual ? mpart.p : nullptr;
    const int per_sm = mixed ? kMinBlocks : 2;
    const unsigned grid = static_cast<unsigned>(
        std::min<int64_t>(pl.n_items, per_sm * static_cast<int64_t>(std::max(1, ctx->sm_count))));
    ctx->mark(Context::kSweepBegin);
    if (pl.n_items > 0) {
        if (mixed && p.kernel == BLTC_KERNEL_YUKAWA) {
            BLTC_CUDA(cudaFuncSetAttribute(k_sweep_hermite_mixed<BLTC_KERNEL_YUKAWA>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmem));
            k_sweep_hermite_mixed<BLTC_KERNEL_YUKAWA><<<grid, kThreads, kMixedSmem, s>>>(a); ++ctx->launches;
        } else if (mixed) {
            BLTC_CUDA(cudaFuncSetAttribute(k_sweep_hermite_mixed<BLTC_KERNEL_COULOMB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmem));
            k_sweep_hermite_mixed<BLTC_KERNEL_COULOMB><<<grid, kThreads, kMixedSmem, s>>>(a); ++ctx->launches;
        } else if (p.kernel == BLTC_KERNEL_YUKAWA) {
            k_sweep_hermite<BLTC_KERNEL_YUKAWA><<<grid, kThreads, 0, s>>>(a); ++ctx->launches;
        } else {
            k_sweep_hermite<BLTC_KERNEL_COULOMB><<<grid, kThreads, 0, s>>>(a); ++ctx->launches;
        }
        BLTC_LAUNCH_CHECK("sweep hermite");
    }
    ctx->mark(Context::kSweepEnd);
    k_finalize<<<static_cast<unsigned>(L->n_batches), 256, 0, s>>>(
        bt->leaves.p, bt->begin.p, bt->count.p, bt->perm.p, pl.n_chunks.p, pl.part_off.p,
        partials.p, L->dir_off.p, pl.dir_sel.p, a.dir_moff, a.mpart, phi, nullptr); ++ctx->launches;
    BLTC_LAUNCH_CHECK("finalize hermite");
    ctx->mark(Context::kEnd);
}

// The finalize of one request whose items have all run (the serving engine's launches).
void launch_finalize(Context* ctx, const Lists* L, const Tree* bt, const double* partials,
                     const float* mpart, double* phi) {
    const Plan& pl = L->plan;
    k_finalize<<<static_cast<unsigned>(L->n_batches), 256, 0, ctx->stream>>>(
        bt->leaves.p, bt->begin.p, bt->count.p, bt->perm.p, pl.n_chunks.p, pl.part_off.p, partials,
        L->dir_off.p, pl.dir_sel.p, pl.mutual ? pl.dir_moff.p : nullptr, pl.mutual ? mpart : nullptr, phi,
        nullptr);
    ++ctx->launches;
    BLTC_LAUNCH_CHECK("finalize multi");
}

}  // namespace bltc
