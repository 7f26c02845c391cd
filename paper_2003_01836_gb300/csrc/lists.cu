// lists.cu -- A1: interaction lists of every target batch (Algorithm 1, Eq. 13).
//
// For each batch B (leaf of the batch tree, DFS order) one warp walks ComputePotential from
// the root of the source tree with an explicit stack, children pushed in reverse so that
// they are visited in stored order, exactly like the recursion:
//   MAC passes ((r_B + r_C)/R < theta and (n+1)^3 < N_C)        -> approximation list
//   geometric test fails ((r_B + r_C)/R not < theta): leaf       -> direct list
//                                                     otherwise  -> the children
//   geometric test passes but (n+1)^3 >= N_C                      -> direct list (whole C)
// A first pass counts, a scan makes CSR offsets, a second pass fills the ids.  The MAC is
// FP64 with IEEE-rounded intrinsics (no fused multiply-add; also --fmad=false), so the
// lists are bit-identical to any other implementation of the same arithmetic.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace bltc {
namespace {

constexpr int kThreads = 64;   // two warps (two batches) per block

struct ListArgs {
    const int32_t* b_leaves;
    const double* b_center;
    const double* b_radius;
    const int32_t* s_count;
    const int32_t* s_nch;
    const int32_t* s_child;
    const double* s_center;
    const double* s_radius;
    int64_t n_batches;
    double theta;
    double theta2;           // theta * theta
    int64_t P;
    int32_t* stack;          // n_batches * stack_cap
    int32_t stack_cap;
    int32_t* app_cnt;        // pass 0
    int32_t* dir_cnt;
    const int32_t* app_off;  // pass 1
    const int32_t* dir_off;
    int32_t* app_ids;
    int32_t* dir_ids;
    int32_t* overflow;
};

enum : int { kApprox = 0, kDirect = 1, kRecurse = 2 };

// Algorithm 1's decision for batch B (centre cb, radius rB) and cluster C.
__device__ __forceinline__ int classify(const ListArgs& a, double cbx, double cby, double cbz,
                                        double rB, int C) {
    const double dx = __dsub_rn(cbx, a.s_center[3 * C]);
    const double dy = __dsub_rn(cby, a.s_center[3 * C + 1]);
    const double dz = __dsub_rn(cbz, a.s_center[3 * C + 2]);
    const double R2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double rs = __dadd_rn(rB, a.s_radius[C]);
    // (r_B + r_C)/R < theta decided from squares when far from the boundary (each side
    // carries a relative rounding error below 1e-15, so a 1e-10 margin cannot flip the
    // decision); otherwise, and for R = 0 or non-finite values, the literal IEEE division
    // and square root of the reading are evaluated.
    const double lhs = __dmul_rn(rs, rs), rhs = __dmul_rn(a.theta2, R2);
    const bool fast = rhs > 1e-290 && rhs < 1e300 && lhs < 1e300;   // normal range
    bool geometric_ok;
    if (fast && lhs < __dmul_rn(rhs, 1.0 - 1e-10))
        geometric_ok = true;
    else if (fast && lhs > __dmul_rn(rhs, 1.0 + 1e-10))
        geometric_ok = false;
    else
        geometric_ok = __ddiv_rn(rs, __dsqrt_rn(R2)) < a.theta;
    const bool size_ok = a.P < static_cast<int64_t>(a.s_count[C]);
    if (geometric_ok && size_ok) return kApprox;
    if (!geometric_ok) return a.s_nch[C] == 0 ? kDirect : kRecurse;
    return kDirect;       // the ratio passes but (n+1)^3 >= N_C: the whole cluster directly
}

// One warp per batch.  The stack holds (cluster, decision); expanding a cluster decides all
// of its children at once (one lane each) and pushes them in reverse so they pop in stored
// order, which reproduces the recursion's visit order exactly.
template <bool kFill>
__global__ void k_lists(ListArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t b = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (b >= a.n_batches) return;
    const int32_t B = a.b_leaves[b];
    if (B < 0) {                       // no batch (beyond the count of a tree sized on the device)
        if (!kFill && lane == 0) a.app_cnt[b] = a.dir_cnt[b] = 0;
        return;
    }
    // entries beyond the batch's range are not written (sized on the device, the offsets are
    // clamped to the capacities, so a batch may get fewer slots than it has entries)
    const int32_t app_end = kFill ? a.app_off[b + 1] - a.app_off[b] : 0;
    const int32_t dir_end = kFill ? a.dir_off[b + 1] - a.dir_off[b] : 0;
    const double cbx = a.b_center[3 * B], cby = a.b_center[3 * B + 1], cbz = a.b_center[3 * B + 2];
    const double rB = a.b_radius[B];
    int2* st = reinterpret_cast<int2*>(a.stack) + b * a.stack_cap;
    int sp = 0;
    if (lane == 0) st[0] = make_int2(0, classify(a, cbx, cby, cbz, rB, 0));
    sp = 1;
    __syncwarp();
    int32_t na = 0, nd = 0;
    int32_t* app = kFill ? a.app_ids + a.app_off[b] : nullptr;
    int32_t* dir = kFill ? a.dir_ids + a.dir_off[b] : nullptr;
    bool overflow = false;
    while (sp > 0) {
        const int2 top = st[--sp];
        if (top.y == kApprox) {
            if (kFill && lane == 0 && na < app_end) app[na] = top.x;
            ++na;
        } else if (top.y == kDirect) {
            if (kFill && lane == 0 && nd < dir_end) dir[nd] = top.x;
            ++nd;
        } else {
            const int k = a.s_nch[top.x];
            if (sp + k > a.stack_cap) {
                overflow = true;
                break;
            }
            if (lane < k) {
                const int c = a.s_child[8 * top.x + lane];
                st[sp + (k - 1 - lane)] = make_int2(c, classify(a, cbx, cby, cbz, rB, c));
            }
            sp += k;
            __syncwarp();
        }
    }
    if (lane == 0) {
        if (overflow) atomicExch(a.overflow, 1);
        if (!kFill) {
            a.app_cnt[b] = na;
            a.dir_cnt[b] = nd;
        }
    }
}

__global__ void k_append_total(int32_t* off, int64_t n, const int32_t* total) {
    off[n] = *total;
}

__global__ void k_raise_if(const int32_t* src, int32_t* flag) {
    if (*src) atomicOr(flag, 1);
}

// Sized on the device: offsets clamped to the capacity, so that every batch's range lies in
// the id array; a total beyond it raises the flag.
__global__ void k_clamp_offsets(int32_t* off, int64_t n, int64_t cap, int32_t* cap_flag) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i > n) return;
    if (off[i] > cap) {
        off[i] = static_cast<int32_t>(cap);
        if (i == n) atomicOr(cap_flag, 1);
    }
}

// Copies the list entries of the selected batches (one block per batch) to their places in
// the new CSR arrays.
__global__ void k_gather_lists(const int32_t* __restrict__ sel, int64_t n_sel,
                               const int32_t* __restrict__ off_old, const int32_t* __restrict__ ids_old,
                               const int32_t* __restrict__ off_new, int32_t* __restrict__ ids_new) {
    for (int64_t i = blockIdx.x; i < n_sel; i += gridDim.x) {
        const int b = sel[i];
        const int a0 = off_old[b], len = off_old[b + 1] - a0, o = off_new[b];
        for (int k = threadIdx.x; k < len; k += blockDim.x) ids_new[o + k] = ids_old[a0 + k];
    }
}

}  // namespace

void build_lists(Context* ctx, const Tree* bt, const Tree* st, double theta, int degree,
                 Lists* out, const Caps* caps) {
    require(degree >= 1 && degree <= BLTC_MAX_DEGREE, "lists: degree out of range");
    require(theta >= 0.0 && theta < 1.0, "lists: theta must satisfy 0 <= theta < 1");
    cudaStream_t s = ctx->stream;
    const int64_t nb = bt->n_leaves;
    const int64_t n1 = degree + 1;
    out->ctx = ctx;
    out->serial = ctx->next_serial++;
    out->bt = bt;
    out->st = st;
    out->theta = theta;
    out->degree = degree;
    out->n_batches = nb;

    ListArgs a{};
    a.b_leaves = bt->leaves.p;
    a.b_center = bt->center.p;
    a.b_radius = bt->radius.p;
    a.s_count = st->count.p;
    a.s_nch = st->nch.p;
    a.s_child = st->child.p;
    a.s_center = st->center.p;
    a.s_radius = st->radius.p;
    a.n_batches = nb;
    a.theta = theta;
    a.theta2 = theta * theta;
    a.P = n1 * n1 * n1;
    a.stack_cap = 7 * st->n_levels + 8;
    DBuf<int32_t> stack(ctx, 2 * nb * a.stack_cap);     // int2 entries
    DBuf<int32_t> cnt(ctx, 2 * nb), flags(ctx, 4);
    out->app_off = DBuf<int32_t>(ctx, nb + 1);
    out->dir_off = DBuf<int32_t>(ctx, nb + 1);
    a.stack = stack.p;
    a.app_cnt = cnt.p;
    a.dir_cnt = cnt.p + nb;
    a.overflow = flags.p + 2;
    if (caps) require(st->caps == caps && bt->caps != nullptr, "lists: trees not sized on the device");
    BLTC_CUDA(cudaMemsetAsync(flags.p, 0, 4 * sizeof(int32_t), s));
    k_lists<false><<<grid_for(32 * nb, kThreads), kThreads, 0, s>>>(a); ++ctx->launches;
    BLTC_LAUNCH_CHECK("lists count");
    exclusive_scan_i32(ctx, a.app_cnt, out->app_off.p, nb, flags.p);
    exclusive_scan_i32(ctx, a.dir_cnt, out->dir_off.p, nb, flags.p + 1);
    k_append_total<<<1, 1, 0, s>>>(out->app_off.p, nb, flags.p); ++ctx->launches;
    k_append_total<<<1, 1, 0, s>>>(out->dir_off.p, nb, flags.p + 1); ++ctx->launches;
    if (caps) {
        // entry counts stay in device memory; the fill writes only batches that fit
        out->caps = caps;
        out->n_app = caps->app;
        out->n_dir = caps->dir;
        out->app_ids = DBuf<int32_t>(ctx, caps->app);
        out->dir_ids = DBuf<int32_t>(ctx, caps->dir);
        k_raise_if<<<1, 1, 0, s>>>(flags.p + 2, caps->flag); ++ctx->launches;   // stack overflow
        out->dcount = std::move(flags);
        k_clamp_offsets<<<grid_for(nb + 1, 256), 256, 0, s>>>(out->app_off.p, nb, caps->app, caps->flag); ++ctx->launches;
        k_clamp_offsets<<<grid_for(nb + 1, 256), 256, 0, s>>>(out->dir_off.p, nb, caps->dir, caps->flag); ++ctx->launches;
        a.app_off = out->app_off.p;
        a.dir_off = out->dir_off.p;
        a.app_ids = out->app_ids.p;
        a.dir_ids = out->dir_ids.p;
        k_lists<true><<<grid_for(32 * nb, kThreads), kThreads, 0, s>>>(a); ++ctx->launches;
        BLTC_LAUNCH_CHECK("lists fill");
        return;
    }
    const int32_t* w = reinterpret_cast<const int32_t*>(ctx->read_words(flags.p, 2));
    const int32_t n_app = w[0], n_dir = w[1], overflow = w[2];
    if (overflow) throw Error(BLTC_ERR_CUDA, "lists: traversal stack overflow");
    out->n_app = n_app;
    out->n_dir = n_dir;
    out->app_ids = DBuf<int32_t>(ctx, n_app);
    out->dir_ids = DBuf<int32_t>(ctx, n_dir);
    a.app_off = out->app_off.p;
    a.dir_off = out->dir_off.p;
    a.app_ids = out->app_ids.p;
    a.dir_ids = out->dir_ids.p;
    k_lists<true><<<grid_for(32 * nb, kThreads), kThreads, 0, s>>>(a); ++ctx->launches;
    BLTC_LAUNCH_CHECK("lists fill");
}

// The lists of some batches only: every other batch keeps an empty list (its targets get
// phi = 0 from an evaluation).  Batches are listed in increasing order.
void select_lists(Context* ctx, const Lists* L, const int32_t* sel, int64_t n_sel, Lists* out) {
    const int64_t nb = L->n_batches;
    require(n_sel >= 0 && (n_sel == 0 || sel != nullptr), "select: batches is NULL");
    for (int64_t i = 0; i < n_sel; ++i) {
        require(sel[i] >= 0 && sel[i] < nb, "select: batch index out of range");
        require(i == 0 || sel[i] > sel[i - 1], "select: batches must be strictly increasing");
    }
    cudaStream_t s = ctx->stream;
    std::vector<int32_t> ha(nb + 1), hd(nb + 1), na(nb + 1, 0), nd(nb + 1, 0);
    BLTC_CUDA(cudaMemcpyAsync(ha.data(), L->app_off.p, sizeof(int32_t) * (nb + 1), cudaMemcpyDeviceToHost, s));
    BLTC_CUDA(cudaMemcpyAsync(hd.data(), L->dir_off.p, sizeof(int32_t) * (nb + 1), cudaMemcpyDeviceToHost, s));
    BLTC_CUDA(cudaStreamSynchronize(s));
    std::vector<char> on(nb, 0);
    for (int64_t i = 0; i < n_sel; ++i) on[sel[i]] = 1;
    for (int64_t b = 0; b < nb; ++b) {
        na[b + 1] = na[b] + (on[b] ? ha[b + 1] - ha[b] : 0);
        nd[b + 1] = nd[b] + (on[b] ? hd[b + 1] - hd[b] : 0);
    }
    out->ctx = ctx;
    out->serial = ctx->next_serial++;
    out->bt = L->bt;
    out->st = L->st;
    out->theta = L->theta;
    out->degree = L->degree;
    out->n_batches = nb;
    out->n_app = na[nb];
    out->n_dir = nd[nb];
    out->app_off = DBuf<int32_t>(ctx, nb + 1);
    out->dir_off = DBuf<int32_t>(ctx, nb + 1);
    out->app_ids = DBuf<int32_t>(ctx, out->n_app);
    out->dir_ids = DBuf<int32_t>(ctx, out->n_dir);
    DBuf<int32_t> dsel(ctx, n_sel);
    BLTC_CUDA(cudaMemcpyAsync(out->app_off.p, na.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, s));
    BLTC_CUDA(cudaMemcpyAsync(out->dir_off.p, nd.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, s));
    if (n_sel > 0) {
        BLTC_CUDA(cudaMemcpyAsync(dsel.p, sel, sizeof(int32_t) * n_sel, cudaMemcpyHostToDevice, s));
        const unsigned g = static_cast<unsigned>(std::min<int64_t>(n_sel, 65535));
        k_gather_lists<<<g, 256, 0, s>>>(dsel.p, n_sel, L->app_off.p, L->app_ids.p, out->app_off.p,
                                         out->app_ids.p);
        ++ctx->launches;
        BLTC_LAUNCH_CHECK("select approximation lists");
        k_gather_lists<<<g, 256, 0, s>>>(dsel.p, n_sel, L->dir_off.p, L->dir_ids.p, out->dir_off.p,
                                         out->dir_ids.p);
        ++ctx->launches;
        BLTC_LAUNCH_CHECK("select direct lists");
    }
    // the host arrays above are read by the copies: wait for them before they go
    BLTC_CUDA(cudaStreamSynchronize(s));
}

}  // namespace bltc
