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
    for (int e = 0; e < ne; ++e) {
        const int64_t c = e < na ? nb * a.P : dir_cost(a, d0 + e - na, nb);
        if (acc > 0 && acc + c > a.cut) {
            if (kFill) out[chunk] = make_int4(static_cast<int>(b), start, e, chunk);
            ++chunk;
            start = e;
            acc = 0;
        }
        acc += c;
    }
    if (kFill) out[chunk] = make_int4(static_cast<int>(b), start, ne, chunk);
    ++chunk;
    if (!kFill) {
        a.n_chunks[b] = chunk;
        a.part_len[b] = chunk * nb;
    }
}

// Interaction count of each item (for longest-first ordering).
__global__ void k_item_costs(PlanArgs a, const int4* __restrict__ items, int64_t n_items,
                             int64_t* cost, const int32_t* n_items_dev) {
    if (n_items_dev) {
        // sized on the device: unwritten items follow an exceeded capacity (nothing runs then)
        if (*a.cap_flag) return;
        if (*n_items_dev < n_items) n_items = *n_items_dev;
    }
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n_items) return;
    const int4 it = items[i];
    const int b = it.x;
    const int64_t nb = a.b_count[a.b_leaves[b]];
    const int a0 = a.app_off[b], na = a.app_off[b + 1] - a0, d0 = a.dir_off[b];
    int64_t c = 0;
    for (int e = it.y; e < it.z; ++e) c += e < na ? nb * a.P : dir_cost(a, d0 + e - na, nb);
    cost[i] = c;
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

// out[0]: direct interactions, out[1]: approximation interactions, out[2]: direct kernel
// evaluations (skipped mutual entries excluded), out[3]: the sweep's cost in target slots
// (each batch's targets padded to its groups' passes, groups_for) times sources, a mutual
// owner's entry weighted 5/4 for its second accumulation.
__global__ void k_counts(const int32_t* b_leaves, const int32_t* b_count, const int32_t* s_count,
                         const int32_t* app_off, const int32_t* dir_off, const int32_t* dir_ids,
                         const uint8_t* dir_sel, int64_t n_batches, int64_t P, unsigned long long* out) {
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
    const int w = kThreads / groups_for(static_cast<int>(nb)) * kT;
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

// The persistent sweep's queue counter: the first real item, or the capacity when the setup
// exceeded a capacity (the sweep then runs nothing and the solve is redone on the host path).
__global__ void k_counter_start(unsigned int* counter, const int32_t* __restrict__ start,
                                const int32_t* __restrict__ stop, int64_t cap) {
    *counter = *stop ? static_cast<unsigned int>(cap) : static_cast<unsigned int>(*start);
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
    k_chunks<true><<<grid_for(L->n_batches, 128), 128, 0, s>>>(a); ++ctx->launches;
    k_item_costs<<<grid_for(cap, 256), 256, 0, s>>>(a, raw.p, cap, icost.p, n_dev); ++ctx->launches;
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

void build_plan(Context* ctx, Lists* L, int degree, bool mutual) {
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
    if (caps) {
        // the cut follows from the total cost in device memory
        a.total_dev = reinterpret_cast<const unsigned long long*>(words.p);
        a.cut_div = blocks * kItemsPerBlock;
        pl.mpart_len = pl.mutual ? std::max<int64_t>(1, caps->mpart_len) : 0;
    } else {
        const int64_t* w0 = ctx->read_words(words.p, 4);
        const int64_t total = w0[0];
        if (pl.mutual) pl.mpart_len = w0[3];
        a.cut = std::max<int64_t>(total / (blocks * kItemsPerBlock), int64_t(1) << 20);
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
        return;
    }
    const int64_t* w = ctx->read_words(words.p, 3);
    pl.n_items = *reinterpret_cast<const int32_t*>(w + 1);
    pl.partial_len = w[2];
    pl.items = DBuf<int4>(ctx, pl.n_items);
    a.item_off = item_off.p;
    a.items = pl.items.p;
    k_chunks<true><<<grid_for(nb, 128), 128, 0, s>>>(a); ++ctx->launches;
    BLTC_LAUNCH_CHECK("plan items");
    // Longest-first order (LPT): the persistent sweep takes items in queue order, so the
    // short ones fill the gaps at the end.  The order does not change any result (each item
    // writes its own partials); ties keep batch order (stable sort).
    if (pl.n_items > 1) {
        DBuf<int64_t> icost(ctx, pl.n_items);
        k_item_costs<<<grid_for(pl.n_items, 256), 256, 0, s>>>(a, pl.items.p, pl.n_items, icost.p, nullptr); ++ctx->launches;
        BLTC_LAUNCH_CHECK("plan costs");
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
    pl.valid = true;
}

static void check_eval(const Lists* L, const Tree* bt, const Tree* st, const bltc_params& p,
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

static SweepArgs make_args(Context* ctx, const Lists* L, const Tree* bt, const Tree* st,
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
    return a;
}


void prepare_plan(Context* ctx, Lists* L, int degree, int precision) {
    const bool mutual = precision == BLTC_PRECISION_MIXED && L->bt == L->st;
    if (!L->plan.valid || L->plan.degree != degree || L->plan.mutual != (mutual && L->n_dir > 0))
        build_plan(ctx, L, degree, mutual);
}

void evaluate(Context* ctx, Lists* L, const Tree* bt, const Tree* st, const bltc_params& p,
              double* phi) {
    check_eval(L, bt, st, p, phi);
    prepare_plan(ctx, L, p.degree, p.precision);
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
    prepare_plan(ctx, L, L->degree, p.precision);
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
    cudaEvent_t done = nullptr;
    bool used = false;
};

MultiSweep::MultiSweep(Context* ctx) : ctx_(ctx) {
    for (int i = 0; i < 2; ++i) {
        slots_.emplace_back(new Slot());
        BLTC_CUDA(cudaEventCreateWithFlags(&slots_.back()->done, cudaEventDisableTiming));
    }
}

MultiSweep::~MultiSweep() {
    for (auto& sl : slots_) {
        if (sl->done) {
            cudaEventSynchronize(sl->done);
            cudaEventDestroy(sl->done);
        }
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
    if (!job.L->plan.valid || job.L->plan.degree != job.p.degree ||
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
    const int64_t cap = kMinBlocks * static_cast<int64_t>(std::max(1, ctx_->sm_count));
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
        if (sl.used) BLTC_CUDA(cudaEventSynchronize(sl.done));     // its previous slice has run
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
        k_finalize<<<static_cast<unsigned>(jb->j.L->n_batches), 256, 0, s>>>(
            jb->j.bt->leaves.p, jb->j.bt->begin.p, jb->j.bt->count.p, jb->j.bt->perm.p, pl.n_chunks.p,
            pl.part_off.p, jb->partials.p, jb->j.L->dir_off.p, pl.dir_sel.p,
            pl.mutual ? pl.dir_moff.p : nullptr, pl.mutual ? jb->mpart.p : nullptr, jb->j.phi, nullptr);
        ++ctx_->launches;
        BLTC_LAUNCH_CHECK("finalize multi");
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

static void counts(Context* ctx, const Lists* L, const uint8_t* dir_sel, int64_t* out4) {
    DBuf<int64_t> w(ctx, 4);
    BLTC_CUDA(cudaMemsetAsync(w.p, 0, 4 * sizeof(int64_t), ctx->stream));
    const int64_t np1 = L->degree + 1;
    k_counts<<<grid_for(L->n_batches, 128), 128, 0, ctx->stream>>>(
        L->bt->leaves.p, L->bt->count.p, L->st->count.p, L->app_off.p, L->dir_off.p,
        L->dir_ids.p, dir_sel, L->n_batches, np1 * np1 * np1, reinterpret_cast<unsigned long long*>(w.p)); ++ctx->launches;
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

int64_t plan_evaluations(Context* ctx, Lists* L, int degree, int precision) {
    require(degree == L->degree, "evaluations: the lists were built for another degree");
    prepare_plan(ctx, L, degree, precision);
    int64_t r[4];
    counts(ctx, L, L->plan.dir_sel.p, r);
    return r[1] + r[2];
}

int64_t plan_slot_cost(Context* ctx, Lists* L, int degree, int precision) {
    require(degree == L->degree, "cost: the lists were built for another degree");
    prepare_plan(ctx, L, degree, precision);
    int64_t r[4];
    counts(ctx, L, L->plan.dir_sel.p, r);
    return r[3];
}

}  // namespace bltc
