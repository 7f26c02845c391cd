// plan.cu -- the sweep's work plan: per direct entry the self-pair, close-pair and mutual-pair
// flags, per batch the cost and the cut of its list into work items of about equal interaction
// count, the items' longest-first order, and the partial and mutual-row layout (Sec. III-B's
// batch-cluster work, arranged for one persistent launch).  Built once per list set and degree,
// host-driven (counts read back, items sorted on the host) or sized on the device.
#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "sweep_device.cuh"

namespace bltc {
namespace {

using namespace sweepdev;

// ---- work plan ------------------------------------------------------------------------

struct PlanArgs {
    const int32_t* b_leaves;
    const int32_t* b_count;
    const int32_t* s_count;
    const int32_t* app_off;
    const int32_t* dir_off;
    const int32_t* dir_ids;
    int64_t n_batches;
    int64_t P;
    int64_t cut;                 // target interactions per item
    int64_t* cost;               // per batch (pass 0)
    unsigned long long* total;
    int32_t* n_chunks;           // per batch
    int64_t* part_len;           // per batch: n_chunks * nb
    const int32_t* item_off;     // pass 2
    int4* items;
    int64_t* icost;              // pass 2: per item its interaction count (the queue order)
    // boxes for the self-pair test
    const double* b_lo;
    const double* b_hi;
    const double* b_center;
    const double* s_lo;
    const double* s_hi;
    uint8_t* dir_sel;
    float* dir_tau2;
    // mutual pairs
    const int32_t* s_nch;
    const int32_t* lidx;         // source node -> batch index (leaves; batches = sources), or -1
    int32_t* partner;            // per direct entry: the partner's entry for B, or -1
    int64_t* mlen;               // per direct entry: mutual row length (owners only)
    const int64_t* moff_e;       // per direct entry: exclusive scan of mlen
    int64_t* dir_moff;
    // sized on the device (else null / unbounded): the direct entry count, the total cost from
    // which the item cut is derived, the item capacity and the overflow flag
    const int32_t* n_dir_dev;
    const unsigned long long* total_dev;
    int64_t cut_div;
    int64_t item_cap;
    int32_t* cap_flag;
};

__device__ __forceinline__ int64_t dir_count(const PlanArgs& a, int64_t n_dir) {
    return a.n_dir_dev && *a.n_dir_dev < n_dir ? *a.n_dir_dev : n_dir;
}

// The batch owning direct entry e: the last b with dir_off[b] <= e.
__device__ __forceinline__ int64_t batch_of_entry(const PlanArgs& a, int64_t e) {
    int64_t lo = 0, hi = a.n_batches;
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (a.dir_off[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// Cost of direct entry e of a batch of nb targets in the mixed sweep: skipped entries cost
// nothing, mutual owners carry the partner's side too.
__device__ __forceinline__ int64_t dir_cost(const PlanArgs& a, int64_t e, int64_t nb) {
    const int64_t c = nb * static_cast<int64_t>(a.s_count[a.dir_ids[e]]);
    if (!a.dir_sel) return c;
    const uint8_t sel = a.dir_sel[e];
    return (sel & kSelSkip) ? 0 : ((sel & kSelMutual) ? c + c / 4 : c);
}

// Marks the direct entries where the mixed sweep must test r^2 == 0.  A target t of batch B
// and a source s of cluster C enter the sweep as fp32(t - c_B) and fp32(s - c_B); each
// rounding moves a coordinate by at most half an FP32 ulp of M, the largest |coordinate -
// c_B| over both boxes in that dimension.  If the boxes are separated in some dimension by
// more than M * 2^-20 (eight ulps) and by more than 1e-18 (so that the squared difference
// stays a normal float), every such pair has a non-zero FP32 difference there, r^2 > 0, and
// the test can be skipped.  Everything else (in particular a batch against itself) keeps
// the test.
__global__ void k_dir_flags(PlanArgs a, int64_t n_dir) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= dir_count(a, n_dir)) return;
    const int B = a.b_leaves[batch_of_entry(a, e)];
    const int C = a.dir_ids[e];
    bool separated = false;
    double Mmax = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double bl = a.b_lo[3 * B + d], bh = a.b_hi[3 * B + d];
        const double cl = a.s_lo[3 * C + d], ch = a.s_hi[3 * C + d];
        const double c = a.b_center[3 * B + d];
        const double gap = fmax(cl - bh, bl - ch);
        const double M = fmax(fmax(fabs(bl - c), fabs(bh - c)), fmax(fabs(cl - c), fabs(ch - c)));
        if (gap > M * 9.5367431640625e-07 && gap > 1e-18) separated = true;
        Mmax = fmax(Mmax, M);
    }
    // Pairs closer than tau = M/64 are recomputed in FP64 by the mixed sweep (their FP32
    // relative error would exceed about 2^-23 * 64 * sqrt(3) ~ 1.3e-5).  Only entries whose
    // boxes come within 1.01 tau of each other can hold such pairs.
    const double tau = Mmax * 0.015625;
    double d2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double gap = fmax(fmax(a.s_lo[3 * C + d] - a.b_hi[3 * B + d], a.b_lo[3 * B + d] - a.s_hi[3 * C + d]), 0.0);
        d2 += gap * gap;
    }
    const bool close = d2 <= 1.0201 * tau * tau;
    a.dir_sel[e] = static_cast<uint8_t>((separated ? 0 : 1) | (close ? 2 : 0));
    a.dir_tau2[e] = static_cast<float>(tau * tau);
}

// Mutual pairs (batches = sources, same tree): leaf C in batch b's direct list whose own
// batch b2 has b's leaf in its direct list.  The entry of the smaller batch index owns the
// pair (bit kSelMutual) and computes both sides; the other is skipped (kSelSkip).  Lists are
// in DFS order, i.e. sorted by node id, so the partner entry is found by binary search.
__global__ void k_leaf_index(PlanArgs a, int32_t* lidx) {
    const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b < a.n_batches && a.b_leaves[b] >= 0) lidx[a.b_leaves[b]] = static_cast<int32_t>(b);
}

__global__ void k_mutual_mark(PlanArgs a, int64_t n_dir) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= dir_count(a, n_dir)) return;
    const int64_t b = batch_of_entry(a, e);
    const int A = a.b_leaves[b], C = a.dir_ids[e];
    int32_t partner = -1;
    int64_t len = 0;
    const int b2 = C != A && a.s_nch[C] == 0 ? a.lidx[C] : -1;
    if (b2 >= 0) {
        const int end = a.dir_off[b2 + 1];
        int lo = a.dir_off[b2], hi = end;                     // search A in [lo, hi)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (a.dir_ids[mid] < A) lo = mid + 1; else hi = mid;
        }
        if (lo < end && a.dir_ids[lo] == A) {
            partner = lo;
            if (b < b2) {
                a.dir_sel[e] |= kSelMutual;
                len = a.s_count[C];
            } else {
                a.dir_sel[e] |= kSelSkip;
            }
        }
    }
    a.partner[e] = partner;
    a.mlen[e] = len;
}

__global__ void k_mutual_moff(PlanArgs a, int64_t n_dir) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= dir_count(a, n_dir)) return;
    const uint8_t sel = a.dir_sel[e];
    a.dir_moff[e] = (sel & kSelMutual) ? a.moff_e[e] : ((sel & kSelSkip) ? a.moff_e[a.partner[e]] : -1);
}

__global__ void k_batch_cost(PlanArgs a) {
    const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= a.n_batches) return;
    if (a.b_leaves[b] < 0) {
        a.cost[b] = 0;
        return;
    }
    const int64_t nb = a.b_count[a.b_leaves[b]];
    int64_t c = static_cast<int64_t>(a.app_off[b + 1] - a.app_off[b]) * a.P * nb;
    for (int e = a.dir_off[b]; e < a.dir_off[b + 1]; ++e) c += dir_cost(a, e, nb);
    a.cost[b] = c;
    atomicAdd(a.total, static_cast<unsigned long long>(c));
}

// Greedy cut of a batch's list (approximated clusters first, then direct ones) into items
// of at most `cut` interactions (an item always takes at least one entry).
template <bool kFill>
__global__ void k_chunks(PlanArgs a) {
    const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= a.n_batches) return;
    if (a.b_leaves[b] < 0) {
        if (!kFill) {
            a.n_chunks[b] = 0;
            a.part_len[b] = 0;
        }
        return;
    }
    if (kFill && a.item_off[b] + a.n_chunks[b] > a.item_cap) {
        atomicOr(a.cap_flag, 1);
        return;
    }
    if (a.total_dev) {
        const int64_t t = static_cast<int64_t>(*a.total_dev) / a.cut_div;
        a.cut = t > (int64_t(1) << 20) ? t : (int64_t(1) << 20);
    }
    const int64_t nb = a.b_count[a.b_leaves[b]];
    const int a0 = a.app_off[b], na = a.app_off[b + 1] - a0;
    const int d0 = a.dir_off[b], nd = a.dir_off[b + 1] - d0;
    const int ne = na + nd;
    int chunk = 0, start = 0;
    int64_t acc = 0;
    int4* out = kFill ? a.items + a.item_off[b] : nullptr;
    int64_t* oc = kFill ? a.icost + a.item_off[b] : nullptr;
    for (int e = 0; e < ne; ++e) {
        const int64_t c = e < na ? nb * a.P : dir_cost(a, d0 + e - na, nb);
        if (acc > 0 && acc + c > a.cut) {
            if (kFill) {
                out[chunk] = make_int4(static_cast<int>(b), start, e, chunk);
                oc[chunk] = acc;
            }
            ++chunk;
            start = e;
            acc = 0;
        }
        acc += c;
    }
    if (kFill) {
        out[chunk] = make_int4(static_cast<int>(b), start, ne, chunk);
        oc[chunk] = acc;
    }
    ++chunk;
    if (!kFill) {
        a.n_chunks[b] = chunk;
        a.part_len[b] = chunk * nb;
    }
}

// out[0]: direct interactions, out[1]: approximation interactions, out[2]: direct kernel
// evaluations (skipped mutual entries excluded), out[3]: the sweep's cost in target slots
// (each batch's targets padded to its groups' passes, groups_for) times sources, a mutual
// owner's entry weighted 5/4 for its second accumulation.
__global__ void k_counts(const int32_t* b_leaves, const int32_t* b_count, const int32_t* s_count,
                         const int32_t* app_off, const int32_t* dir_off, const int32_t* dir_ids,
                         const uint8_t* dir_sel, int64_t n_batches, int64_t P, int g_max,
                         unsigned long long* out) {
    const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= n_batches) return;
    const int64_t nb = b_count[b_leaves[b]];
    int64_t d = 0, de = 0, dw = 0;
    for (int e = dir_off[b]; e < dir_off[b + 1]; ++e) {
        const int64_t c = s_count[dir_ids[e]];
        d += c;
        if (!dir_sel || !(dir_sel[e] & kSelSkip)) {
            de += c;
            dw += (dir_sel && (dir_sel[e] & kSelMutual)) ? c + c / 4 : c;
        }
    }
    const int64_t app = static_cast<int64_t>(app_off[b + 1] - app_off[b]) * P;
    const int w = kThreads / groups_for(static_cast<int>(nb), g_max) * kT;
    const int64_t slots = (nb + w - 1) / w * w;
    atomicAdd(&out[0], static_cast<unsigned long long>(d * nb));
    atomicAdd(&out[1], static_cast<unsigned long long>(app * nb));
    atomicAdd(&out[2], static_cast<unsigned long long>(de * nb));
    atomicAdd(&out[3], static_cast<unsigned long long>((app + dw) * slots));
}

// ---- the plan sized on the device --------------------------------------------------------
//
// Items are placed longest first by a bucket sort on the device: a key per item from its cost
// (four buckets per octave, larger costs first), a histogram, offsets, and a scatter whose order
// within a bucket follows the atomics.  As on the host, the order changes no result (each item
// writes its own partials and rows), only how the persistent sweep's blocks share the work.
// The sorted items occupy the end of the item array, [cap - n, cap), so that the sweep, whose
// queue ends at the capacity, starts its counter at cap - n (cap when a capacity was exceeded:
// no item runs) and stays the same kernel as the host-driven path launches.
constexpr int kBuckets = 256;

__device__ __forceinline__ int cost_bucket(int64_t c) {
    if (c <= 0) return kBuckets - 1;
    const int e = 63 - __clzll(static_cast<unsigned long long>(c));
    const int f = e >= 2 ? static_cast<int>((static_cast<unsigned long long>(c) >> (e - 2)) & 3) : 0;
    const int level = 4 * e + f;              // 0 .. 255, increasing with the cost
    return kBuckets - 1 - level;              // longest first
}

__global__ void k_bucket_hist(const int64_t* __restrict__ cost, const int32_t* __restrict__ n_dev,
                              int64_t cap, int32_t* hist) {
    const int64_t n = min(static_cast<int64_t>(*n_dev), cap);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        atomicAdd(&hist[cost_bucket(cost[i])], 1);
}

// One warp: bucket offsets from cap - n, zero cursors, the sweep's first item, and the checks
// of the plan's totals against their capacities.
__global__ void k_bucket_offsets(int32_t* hist, const int64_t* __restrict__ words, int64_t item_cap,
                                 int64_t partial_cap, int64_t mpart_cap, int32_t* start, int32_t* cap_flag) {
    const int32_t n = reinterpret_cast<const int32_t*>(words + 1)[0];
    const bool over = n > item_cap || words[2] > partial_cap || words[3] > mpart_cap;
    if (threadIdx.x == 0) {
        if (over) atomicOr(cap_flag, 1);
        int64_t o = item_cap - min(static_cast<int64_t>(n), item_cap);
        for (int k = 0; k < kBuckets; ++k) {
            const int32_t h = hist[k];
            hist[kBuckets + k] = static_cast<int32_t>(o);
            hist[2 * kBuckets + k] = 0;
            o += h;
        }
        *start = static_cast<int32_t>(item_cap - min(static_cast<int64_t>(n), item_cap));
    }
}

__global__ void k_bucket_scatter(const int4* __restrict__ raw, const int64_t* __restrict__ cost,
                                 const int32_t* __restrict__ n_dev, int64_t cap, int32_t* hist,
                                 int4* __restrict__ sorted) {
    const int64_t n = min(static_cast<int64_t>(*n_dev), cap);
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int k = cost_bucket(cost[i]);
        sorted[hist[kBuckets + k] + atomicAdd(&hist[2 * kBuckets + k], 1)] = raw[i];
    }
}

}  // namespace

static void build_plan_sized(Context* ctx, Lists* L, PlanArgs a, DBuf<int32_t>& item_off,
                             DBuf<int64_t>& words, int degree) {
    cudaStream_t s = ctx->stream;
    const Caps* caps = L->caps;
    Plan& pl = L->plan;
    const int64_t cap = a.item_cap;
    pl.n_items = cap;
    pl.partial_len = std::max<int64_t>(1, caps->partial_len);
    pl.dwords = std::move(words);
    pl.dstart = DBuf<int32_t>(ctx, 1);
    DBuf<int4> raw(ctx, cap);
    DBuf<int64_t> icost(ctx, cap);
    DBuf<int32_t> hist(ctx, 3 * kBuckets);
    pl.items = DBuf<int4>(ctx, cap);
    const int32_t* n_dev = reinterpret_cast<const int32_t*>(pl.dwords.p + 1);
    a.item_off = item_off.p;
    a.items = raw.p;
    a.icost = icost.p;
    k_chunks<true><<<grid_for(L->n_batches, 128), 128, 0, s>>>(a); ++ctx->launches;
    BLTC_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(int32_t) * kBuckets, s));
    const unsigned g = grid_for(cap, 256, 4 * std::max(1, ctx->sm_count));
    k_bucket_hist<<<g, 256, 0, s>>>(icost.p, n_dev, cap, hist.p); ++ctx->launches;
    k_bucket_offsets<<<1, 32, 0, s>>>(hist.p, pl.dwords.p, cap, pl.partial_len,
                                      pl.mutual ? pl.mpart_len : INT64_MAX, pl.dstart.p, caps->flag); ++ctx->launches;
    k_bucket_scatter<<<g, 256, 0, s>>>(raw.p, icost.p, n_dev, cap, hist.p, pl.items.p); ++ctx->launches;
    BLTC_LAUNCH_CHECK("plan items (sized on the device)");
    pl.h_cost.clear();
    pl.degree = degree;
    pl.valid = true;
}

void build_plan(Context* ctx, Lists* L, int degree, bool mutual, int tile) {
    cudaStream_t s = ctx->stream;
    const int64_t nb = L->n_batches;
    const int64_t np1 = degree + 1;
    const Caps* caps = L->caps;
    Plan& pl = L->plan;
    pl.valid = false;
    PlanArgs a{};
    a.b_leaves = L->bt->leaves.p;
    a.b_count = L->bt->count.p;
    a.s_count = L->st->count.p;
    a.app_off = L->app_off.p;
    a.dir_off = L->dir_off.p;
    a.dir_ids = L->dir_ids.p;
    a.n_batches = nb;
    a.P = np1 * np1 * np1;
    a.item_cap = INT64_MAX;
    if (caps) {
        a.n_dir_dev = L->dcount.p + 1;
        a.cap_flag = caps->flag;
        a.item_cap = std::max<int64_t>(1, caps->items);
    }
    // per direct entry: the self-pair and close-pair flags, then the mutual pairs
    pl.dir_sel = DBuf<uint8_t>(ctx, L->n_dir);
    pl.dir_tau2 = DBuf<float>(ctx, L->n_dir);
    a.dir_tau2 = pl.dir_tau2.p;
    a.b_lo = L->bt->lo.p;
    a.b_hi = L->bt->hi.p;
    a.b_center = L->bt->center.p;
    a.s_lo = L->st->lo.p;
    a.s_hi = L->st->hi.p;
    a.dir_sel = pl.dir_sel.p;
    if (L->n_dir > 0) {
        k_dir_flags<<<grid_for(L->n_dir, 256), 256, 0, s>>>(a, L->n_dir); ++ctx->launches;
    }
    BLTC_LAUNCH_CHECK("plan flags");
    pl.mutual = mutual && L->bt == L->st && L->n_dir > 0;
    pl.mpart_len = 0;
    pl.dir_moff = DBuf<int64_t>();
    // words: [0] total cost, [1] items (int32), [2] partial length, [3] mutual row length
    DBuf<int64_t> cost(ctx, nb), part_len(ctx, nb), words(ctx, 4);
    BLTC_CUDA(cudaMemsetAsync(words.p, 0, 4 * sizeof(int64_t), s));
    if (pl.mutual) {
        const int64_t m = L->st->n_nodes;
        DBuf<int32_t> lidx(ctx, m), partner(ctx, L->n_dir);
        DBuf<int64_t> mlen(ctx, L->n_dir), moff_e(ctx, L->n_dir);
        pl.dir_moff = DBuf<int64_t>(ctx, L->n_dir);
        BLTC_CUDA(cudaMemsetAsync(lidx.p, 0xff, sizeof(int32_t) * m, s));
        if (caps) BLTC_CUDA(cudaMemsetAsync(mlen.p, 0, sizeof(int64_t) * L->n_dir, s));
        a.s_nch = L->st->nch.p;
        a.lidx = lidx.p;
        a.partner = partner.p;
        a.mlen = mlen.p;
        a.moff_e = moff_e.p;
        a.dir_moff = pl.dir_moff.p;
        k_leaf_index<<<grid_for(nb, 256), 256, 0, s>>>(a, lidx.p); ++ctx->launches;
        k_mutual_mark<<<grid_for(L->n_dir, 256), 256, 0, s>>>(a, L->n_dir); ++ctx->launches;
        BLTC_LAUNCH_CHECK("plan mutual");
        exclusive_scan_i64(ctx, mlen.p, moff_e.p, L->n_dir, words.p + 3);
        k_mutual_moff<<<grid_for(L->n_dir, 256), 256, 0, s>>>(a, L->n_dir); ++ctx->launches;
        BLTC_LAUNCH_CHECK("plan mutual rows");
    }
    // costs and items (skipped mutual entries cost nothing)
    a.cost = cost.p;
    a.total = reinterpret_cast<unsigned long long*>(words.p);
    k_batch_cost<<<grid_for(nb, 128), 128, 0, s>>>(a); ++ctx->launches;
    BLTC_LAUNCH_CHECK("plan cost");
    const int64_t blocks = kMinBlocks * static_cast<int64_t>(std::max(1, ctx->sm_count));
    const int64_t per_block = tile_items_per_block(tile);
    if (caps) {
        // the cut follows from the total cost in device memory
        a.total_dev = reinterpret_cast<const unsigned long long*>(words.p);
        a.cut_div = blocks * per_block;
        pl.mpart_len = pl.mutual ? std::max<int64_t>(1, caps->mpart_len) : 0;
    } else {
        const int64_t* w0 = ctx->read_words(words.p, 4);
        const int64_t total = w0[0];
        if (pl.mutual) pl.mpart_len = w0[3];
        a.cut = std::max<int64_t>(total / (blocks * per_block), int64_t(1) << 20);
    }
    pl.n_chunks = DBuf<int32_t>(ctx, nb);
    pl.part_off = DBuf<int64_t>(ctx, nb);
    DBuf<int32_t> item_off(ctx, nb);
    a.n_chunks = pl.n_chunks.p;
    a.part_len = part_len.p;
    k_chunks<false><<<grid_for(nb, 128), 128, 0, s>>>(a); ++ctx->launches;
    BLTC_LAUNCH_CHECK("plan chunks");
    exclusive_scan_i32(ctx, pl.n_chunks.p, item_off.p, nb, reinterpret_cast<int32_t*>(words.p + 1));
    exclusive_scan_i64(ctx, part_len.p, pl.part_off.p, nb, words.p + 2);
    if (caps) {
        build_plan_sized(ctx, L, a, item_off, words, degree);
        pl.tile = tile;
        return;
    }
    const int64_t* w = ctx->read_words(words.p, 3);
    pl.n_items = *reinterpret_cast<const int32_t*>(w + 1);
    pl.partial_len = w[2];
    pl.items = DBuf<int4>(ctx, pl.n_items);
    DBuf<int64_t> icost(ctx, pl.n_items);
    a.item_off = item_off.p;
    a.items = pl.items.p;
    a.icost = icost.p;
    k_chunks<true><<<grid_for(nb, 128), 128, 0, s>>>(a); ++ctx->launches;
    BLTC_LAUNCH_CHECK("plan items");
    // Longest-first order (LPT): the persistent sweep takes items in queue order, so the
    // short ones fill the gaps at the end.  The order does not change any result (each item
    // writes its own partials); ties keep batch order (stable sort).
    if (pl.n_items > 1) {
        std::vector<int4> h_items(static_cast<size_t>(pl.n_items));
        std::vector<int64_t> h_cost(static_cast<size_t>(pl.n_items));
        BLTC_CUDA(cudaMemcpyAsync(h_items.data(), pl.items.p, sizeof(int4) * pl.n_items, cudaMemcpyDeviceToHost, s));
        BLTC_CUDA(cudaMemcpyAsync(h_cost.data(), icost.p, sizeof(int64_t) * pl.n_items, cudaMemcpyDeviceToHost, s));
        BLTC_CUDA(cudaStreamSynchronize(s));
        std::vector<int64_t> order(static_cast<size_t>(pl.n_items));
        for (int64_t i = 0; i < pl.n_items; ++i) order[static_cast<size_t>(i)] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int64_t x, int64_t y) { return h_cost[static_cast<size_t>(x)] > h_cost[static_cast<size_t>(y)]; });
        std::vector<int4> sorted(static_cast<size_t>(pl.n_items));
        for (int64_t i = 0; i < pl.n_items; ++i) sorted[static_cast<size_t>(i)] = h_items[static_cast<size_t>(order[static_cast<size_t>(i)])];
        BLTC_CUDA(cudaMemcpyAsync(pl.items.p, sorted.data(), sizeof(int4) * pl.n_items, cudaMemcpyHostToDevice, s));
        BLTC_CUDA(cudaStreamSynchronize(s));
        pl.h_cost.resize(static_cast<size_t>(pl.n_items));
        for (int64_t i = 0; i < pl.n_items; ++i) pl.h_cost[static_cast<size_t>(i)] = h_cost[static_cast<size_t>(order[static_cast<size_t>(i)])];
    } else {
        pl.h_cost.assign(static_cast<size_t>(pl.n_items), 1);
    }
    pl.degree = degree;
    pl.tile = tile;
    pl.valid = true;
}

void prepare_plan(Context* ctx, Lists* L, int degree, int precision, int tile) {
    const bool mutual = precision == BLTC_PRECISION_MIXED && L->bt == L->st;
    if (!L->plan.valid || L->plan.degree != degree || L->plan.mutual != (mutual && L->n_dir > 0) ||
        L->plan.tile != tile)
        build_plan(ctx, L, degree, mutual, tile);
}

static void counts(Context* ctx, const Lists* L, const uint8_t* dir_sel, int64_t* out4, int g_max = 8) {
    DBuf<int64_t> w(ctx, 4);
    BLTC_CUDA(cudaMemsetAsync(w.p, 0, 4 * sizeof(int64_t), ctx->stream));
    const int64_t np1 = L->degree + 1;
    k_counts<<<grid_for(L->n_batches, 128), 128, 0, ctx->stream>>>(
        L->bt->leaves.p, L->bt->count.p, L->st->count.p, L->app_off.p, L->dir_off.p,
        L->dir_ids.p, dir_sel, L->n_batches, np1 * np1 * np1, g_max, reinterpret_cast<unsigned long long*>(w.p)); ++ctx->launches;
    BLTC_LAUNCH_CHECK("counts");
    const int64_t* r = ctx->read_words(w.p, 4);
    for (int i = 0; i < 4; ++i) out4[i] = r[i];
}

void interaction_counts(Context* ctx, const Lists* L, int64_t* n_dir, int64_t* n_app) {
    int64_t r[4];
    counts(ctx, L, nullptr, r);
    if (n_dir) *n_dir = r[0];
    if (n_app) *n_app = r[1];
}

int64_t plan_evaluations(Context* ctx, Lists* L, int degree, int precision, int tile) {
    require(degree == L->degree, "evaluations: the lists were built for another degree");
    prepare_plan(ctx, L, degree, precision, tile);
    int64_t r[4];
    counts(ctx, L, L->plan.dir_sel.p, r);
    return r[1] + r[2];
}

int64_t plan_slot_cost(Context* ctx, Lists* L, int degree, int precision, int tile) {
    require(degree == L->degree, "cost: the lists were built for another degree");
    prepare_plan(ctx, L, degree, precision, tile);
    int64_t r[4];
    counts(ctx, L, L->plan.dir_sel.p, r, tile_group_cap(tile));
    return r[3];
}

}  // namespace bltc
