// cp.cu -- the cluster-particle variant (future work of Sec. V): the roles of Algorithm 1
// swapped, targets interpolated and sources summed exactly.
//
// For every source batch S (a leaf of the source tree) ComputePotential walks the target
// tree with the MAC of Eq. 13, (r_S + r_T)/R < theta and (n+1)^3 < N_T.  An approximated
// target cluster T accumulates the potential at its Chebyshev points,
//     phihat_T[k] = sum_{S approximating T} sum_{y_j in S} G(t_k, y_j) q_j,
// a direct one the potentials of its targets; each target then adds the interpolant
// sum_k L_k1(x1) L_k2(x2) L_k3(x3) phihat_T[k] (Eq. 4-8, exact hits of Sec. II-C) of every
// cluster holding it, from the root down.
//
// GB300 mapping: both halves are direct sums, so both run on the library's sweep.  The
// lists (the same list builder, batches = source leaves, clusters = target tree) are turned
// around per target: the far half becomes a sweep whose "batches" are the Chebyshev grids of
// the approximated target clusters (a synthetic tree of P points per cluster), the near half
// a sweep over the target leaves with direct lists only.  A last kernel interpolates.  Every
// per-target list is sorted by source batch, so sums run in a fixed order.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace bltc {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxDepth = 128;         // target tree levels the interpolation walks

__global__ void k_cp_total(int32_t* off, int64_t n, const int32_t* total) { off[n] = *total; }

// The source batch owning list entry e (the last b with off[b] <= e).
__device__ __forceinline__ int batch_of(const int32_t* off, int nb, int64_t e) {
    int lo = 0, hi = nb;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// Leaves of target node T: a contiguous range of the DFS-ordered leaf list, found from the
// leaves' first particle positions (ascending).
__device__ __forceinline__ void leaf_range(const int32_t* leaf_begin, int n_leaves, int b0, int b1,
                                           int* i0, int* i1) {
    int lo = 0, hi = n_leaves;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (leaf_begin[mid] < b0) lo = mid + 1; else hi = mid;
    }
    *i0 = lo;
    hi = n_leaves;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (leaf_begin[mid] < b1) lo = mid + 1; else hi = mid;
    }
    *i1 = lo;
}

__global__ void k_leaf_begin(const int32_t* leaves, const int32_t* begin, int n_leaves, int32_t* leaf_begin) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_leaves) leaf_begin[i] = begin[leaves[i]];
}

// Counts, then fills, the per-target lists: far (per target node) and near (per target
// leaf; a direct cluster hands its batch to each of its leaves).
template <bool kFill>
__global__ void k_cp_lists(const int32_t* __restrict__ app_off, const int32_t* __restrict__ app_ids,
                           int64_t n_app, const int32_t* __restrict__ dir_off,
                           const int32_t* __restrict__ dir_ids, int64_t n_dir, int n_batches,
                           const int32_t* __restrict__ s_leaves, const int32_t* __restrict__ t_begin,
                           const int32_t* __restrict__ t_count, const int32_t* __restrict__ leaf_begin,
                           int n_leaves, int32_t* far_cnt, int32_t* near_cnt,
                           const int32_t* __restrict__ far_off, const int32_t* __restrict__ near_off,
                           int32_t* far_ids, int32_t* near_ids) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < n_app) {
        const int b = batch_of(app_off, n_batches, e);
        const int T = app_ids[e];
        const int pos = atomicAdd(&far_cnt[T], 1);
        if (kFill) far_ids[far_off[T] + pos] = s_leaves[b];
    } else if (e < n_app + n_dir) {
        const int64_t d = e - n_app;
        const int b = batch_of(dir_off, n_batches, d);
        const int T = dir_ids[d];
        int i0, i1;
        leaf_range(leaf_begin, n_leaves, t_begin[T], t_begin[T] + t_count[T], &i0, &i1);
        for (int i = i0; i < i1; ++i) {
            const int pos = atomicAdd(&near_cnt[i], 1);
            if (kFill) near_ids[near_off[i] + pos] = s_leaves[b];
        }
    }
}

// Each segment in ascending source-leaf id (= ascending batch, leaves are in DFS order).
__global__ void k_cp_sort(const int32_t* __restrict__ off, int n, int32_t* ids) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t* a = ids + off[i];
    const int m = off[i + 1] - off[i];
    for (int x = 1; x < m; ++x) {
        const int32_t v = a[x];
        int y = x - 1;
        while (y >= 0 && a[y] > v) {
            a[y + 1] = a[y];
            --y;
        }
        a[y + 1] = v;
    }
}

__global__ void k_flag_nonzero(const int32_t* cnt, int64_t n, int32_t* flag) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = cnt[i] > 0 ? 1 : 0;
}

// The approximated target clusters in id order, their index, and their list offsets.
__global__ void k_cp_compact(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                             const int32_t* __restrict__ far_off, int64_t m, int32_t* tlist,
                             int32_t* tidx, int32_t* off_c) {
    const int64_t T = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (T >= m) return;
    if (flag[T]) {
        tlist[pos[T]] = static_cast<int32_t>(T);
        tidx[T] = pos[T];
        off_c[pos[T]] = far_off[T];
    } else {
        tidx[T] = -1;
    }
}

// Chebyshev point k of [lo, hi] (Eq. 6 mapped linearly; s_0 = hi and s_n = lo exactly).
__device__ __forceinline__ double cheb_pt(const double* t, int k, int n, double lo, double hi) {
    if (k == 0) return hi;
    if (k == n) return lo;
    return __dadd_rn(lo, __dmul_rn(__dmul_rn(0.5, __dadd_rn(t[k], 1.0)), __dsub_rn(hi, lo)));
}

// The synthetic batch tree of the far half: one leaf per approximated target cluster, its
// P Chebyshev points as particles (k = (k1 (n+1) + k2)(n+1) + k3), the cluster's box.
__global__ void k_cp_proxy(const int32_t* __restrict__ tlist, int nt_app, const double* __restrict__ lo,
                           const double* __restrict__ hi, const double* __restrict__ center,
                           const double* __restrict__ radius, const double* __restrict__ cheb_t, int np1,
                           double* px, double* py, double* pz, int32_t* perm, int32_t* begin,
                           int32_t* count, int32_t* leaves, int32_t* nch, int32_t* parent,
                           double* plo, double* phi_, double* pc, double* pr) {
    const int i = blockIdx.x;
    const int T = tlist[i];
    const int n = np1 - 1, P = np1 * np1 * np1;
    if (threadIdx.x == 0) {
        begin[i] = i * P;
        count[i] = P;
        leaves[i] = i;
        nch[i] = 0;
        parent[i] = -1;
        pr[i] = radius[T];
        for (int d = 0; d < 3; ++d) {
            plo[3 * i + d] = lo[3 * T + d];
            phi_[3 * i + d] = hi[3 * T + d];
            pc[3 * i + d] = center[3 * T + d];
        }
    }
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        const int k1 = k / (np1 * np1), r = k - k1 * np1 * np1, k2 = r / np1, k3 = r - k2 * np1;
        const int64_t o = static_cast<int64_t>(i) * P + k;
        px[o] = cheb_pt(cheb_t, k1, n, lo[3 * T], hi[3 * T]);
        py[o] = cheb_pt(cheb_t, k2, n, lo[3 * T + 1], hi[3 * T + 1]);
        pz[o] = cheb_pt(cheb_t, k3, n, lo[3 * T + 2], hi[3 * T + 2]);
        perm[o] = static_cast<int32_t>(o);
    }
}

// Interpolation to the targets: per target leaf (a block), for each cluster on its path
// that holds point potentials, root first, the three 1-D Lagrange vectors of the target
// (barycentric, exact hits) contracted with phihat_T.  FP64.
__global__ void __launch_bounds__(256) k_cp_l2p(const int32_t* __restrict__ leaves,
                                                const int32_t* __restrict__ begin,
                                                const int32_t* __restrict__ count,
                                                const int32_t* __restrict__ parent,
                                                const int32_t* __restrict__ perm,
                                                const double* __restrict__ px, const double* __restrict__ py,
                                                const double* __restrict__ pz, const double* __restrict__ lo,
                                                const double* __restrict__ hi, const double* __restrict__ cheb_t,
                                                const int32_t* __restrict__ tidx,
                                                const double* __restrict__ phat, int np1, double* phi) {
    extern __shared__ double l2p_smem[];                 // phihat of one cluster, P values
    __shared__ int chain[kMaxDepth];
    __shared__ int depth;
    __shared__ double s_pts[3 * (BLTC_MAX_DEGREE + 1)];
    const int L = leaves[blockIdx.x];
    const int n = np1 - 1, P = np1 * np1 * np1;
    if (threadIdx.x == 0) {
        int dd = 0;
        for (int v = L; v >= 0 && dd < kMaxDepth; v = parent[v]) chain[dd++] = v;
        depth = dd;
    }
    __syncthreads();
    const int tb = begin[L], nb = count[L];
    // each thread keeps up to 8 targets' sums
    constexpr int U = 8;
    double acc[U];
    for (int t0 = 0; t0 < nb; t0 += U * static_cast<int>(blockDim.x)) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + static_cast<int>(threadIdx.x) + u * static_cast<int>(blockDim.x);
            acc[u] = t < nb ? phi[perm[tb + t]] : 0.0;
        }
        for (int d = depth - 1; d >= 0; --d) {
            const int T = chain[d];
            const int slot = tidx[T];
            if (slot < 0) continue;
            __syncthreads();
            for (int k = threadIdx.x; k < P; k += blockDim.x) l2p_smem[k] = phat[static_cast<int64_t>(slot) * P + k];
            if (threadIdx.x < 3 * np1) {
                const int dim = threadIdx.x / np1, k = threadIdx.x - dim * np1;
                s_pts[threadIdx.x] = cheb_pt(cheb_t, k, n, lo[3 * T + dim], hi[3 * T + dim]);
            }
            __syncthreads();
#pragma unroll 1
            for (int u = 0; u < U; ++u) {
                const int t = t0 + static_cast<int>(threadIdx.x) + u * static_cast<int>(blockDim.x);
                if (t >= nb) continue;
                const double y[3] = {px[tb + t], py[tb + t], pz[tb + t]};
                double a[3][BLTC_MAX_DEGREE + 1];
                for (int dim = 0; dim < 3; ++dim) {
                    const double* s = s_pts + dim * np1;
                    int hit = -1;
                    for (int k = 0; k < np1; ++k)
                        if (hit < 0 && fabs(y[dim] - s[k]) < 2.2250738585072014e-308) hit = k;
                    if (hit >= 0) {
                        for (int k = 0; k < np1; ++k) a[dim][k] = k == hit ? 1.0 : 0.0;
                    } else {
                        double den = 0.0;
                        for (int k = 0; k < np1; ++k) {
                            const double w = ((k == 0 || k == n) ? 0.5 : 1.0) * ((k & 1) ? -1.0 : 1.0);
                            a[dim][k] = w / (y[dim] - s[k]);
                            den += a[dim][k];
                        }
                        for (int k = 0; k < np1; ++k) a[dim][k] /= den;
                    }
                }
                double sum = 0.0;
                for (int k1 = 0; k1 < np1; ++k1)
                    for (int k2 = 0; k2 < np1; ++k2) {
                        const double a12 = a[0][k1] * a[1][k2];
                        const double* row = l2p_smem + (k1 * np1 + k2) * np1;
                        for (int k3 = 0; k3 < np1; ++k3) sum += a12 * a[2][k3] * row[k3];
                    }
                acc[u] += sum;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + static_cast<int>(threadIdx.x) + u * static_cast<int>(blockDim.x);
            if (t < nb) phi[perm[tb + t]] = acc[u];
        }
    }
}

}  // namespace

void solve_device_cp(Context* c, const double* tx, const double* ty, const double* tz, int64_t nt,
                     const double* sx, const double* sy, const double* sz, const double* sq, int64_t ns,
                     const bltc_params& p, double* phi) {
    cudaStream_t s = c->stream;
    const int np1 = p.degree + 1, P = np1 * np1 * np1;
    c->mark(Context::kStart);
    Tree ts, ss;
    build_tree(c, sx, sy, sz, sq, ns, p.batch_size, &ss);           // source batches
    // the same particles with the same leaf size share one tree, so that the near half's
    // mutual leaf pairs are evaluated once (mixed sweep)
    const bool same = tx == sx && ty == sy && tz == sz && nt == ns && p.leaf_size == p.batch_size;
    if (!same) build_tree(c, tx, ty, tz, nullptr, nt, p.leaf_size, &ts);   // target clusters
    Tree& tt = same ? ss : ts;
    require(tt.n_levels <= kMaxDepth, "solve_cp: target tree deeper than 128 levels");
    c->mark(Context::kTrees);
    Lists L;                                                        // per source batch
    build_lists(c, &ss, &tt, p.theta, p.degree, &L);
    c->mark(Context::kLists);
    // modified charges are not used (no source cluster is approximated); mark the source
    // tree as ready for this degree and precision with no slots
    ss.q_degree = p.degree;
    ss.q_precision = p.precision;
    ss.q_lists = 0;
    ss.q_slots = 0;

    // turn the lists around: per target node (far) and per target leaf (near)
    const int64_t m = tt.n_nodes;
    const int nl = static_cast<int>(tt.n_leaves);
    const int nbat = static_cast<int>(L.n_batches);
    DBuf<int32_t> leaf_begin(c, nl), far_cnt(c, m), near_cnt(c, nl), far_off(c, m + 1), near_off(c, nl + 1),
        tot(c, 4);
    k_leaf_begin<<<grid_for(nl, kThreads), kThreads, 0, s>>>(tt.leaves.p, tt.begin.p, nl, leaf_begin.p); ++c->launches;
    BLTC_CUDA(cudaMemsetAsync(far_cnt.p, 0, sizeof(int32_t) * m, s));
    BLTC_CUDA(cudaMemsetAsync(near_cnt.p, 0, sizeof(int32_t) * nl, s));
    const int64_t ne = L.n_app + L.n_dir;
    if (ne > 0) {
        k_cp_lists<false><<<grid_for(ne, kThreads), kThreads, 0, s>>>(
            L.app_off.p, L.app_ids.p, L.n_app, L.dir_off.p, L.dir_ids.p, L.n_dir, nbat, ss.leaves.p,
            tt.begin.p, tt.count.p, leaf_begin.p, nl, far_cnt.p, near_cnt.p, nullptr, nullptr, nullptr,
            nullptr); ++c->launches;
    }
    BLTC_LAUNCH_CHECK("cp count");
    exclusive_scan_i32(c, far_cnt.p, far_off.p, m, tot.p);
    exclusive_scan_i32(c, near_cnt.p, near_off.p, nl, tot.p + 1);
    k_cp_total<<<1, 1, 0, s>>>(far_off.p, m, tot.p); ++c->launches;
    k_cp_total<<<1, 1, 0, s>>>(near_off.p, nl, tot.p + 1); ++c->launches;
    // approximated target clusters, compacted
    DBuf<int32_t> flag(c, m), pos(c, m), tidx(c, m);
    k_flag_nonzero<<<grid_for(m, kThreads), kThreads, 0, s>>>(far_cnt.p, m, flag.p); ++c->launches;
    exclusive_scan_i32(c, flag.p, pos.p, m, tot.p + 2);
    const int32_t* w = reinterpret_cast<const int32_t*>(c->read_words(tot.p, 2));
    const int32_t n_far = w[0], n_near = w[1], nt_app = w[2];
    DBuf<int32_t> far_ids(c, n_far), near_ids(c, n_near), tlist(c, nt_app), off_c(c, nt_app + 1);
    BLTC_CUDA(cudaMemsetAsync(far_cnt.p, 0, sizeof(int32_t) * m, s));
    BLTC_CUDA(cudaMemsetAsync(near_cnt.p, 0, sizeof(int32_t) * nl, s));
    if (ne > 0) {
        k_cp_lists<true><<<grid_for(ne, kThreads), kThreads, 0, s>>>(
            L.app_off.p, L.app_ids.p, L.n_app, L.dir_off.p, L.dir_ids.p, L.n_dir, nbat, ss.leaves.p,
            tt.begin.p, tt.count.p, leaf_begin.p, nl, far_cnt.p, near_cnt.p, far_off.p, near_off.p,
            far_ids.p, near_ids.p); ++c->launches;
    }
    BLTC_LAUNCH_CHECK("cp fill");
    k_cp_sort<<<grid_for(m, 128), 128, 0, s>>>(far_off.p, static_cast<int>(m), far_ids.p); ++c->launches;
    k_cp_sort<<<grid_for(nl, 128), 128, 0, s>>>(near_off.p, nl, near_ids.p); ++c->launches;
    k_cp_compact<<<grid_for(m, kThreads), kThreads, 0, s>>>(flag.p, pos.p, far_off.p, m, tlist.p, tidx.p,
                                                         off_c.p); ++c->launches;
    k_cp_total<<<1, 1, 0, s>>>(off_c.p, nt_app, tot.p); ++c->launches;
    BLTC_LAUNCH_CHECK("cp lists");
    c->mark(Context::kUpward);

    // near half: a sweep over the target leaves with direct lists only
    {
        Lists Ln;
        Ln.ctx = c;
        Ln.serial = c->next_serial++;
        Ln.bt = &tt;
        Ln.st = &ss;
        Ln.theta = p.theta;
        Ln.degree = p.degree;
        Ln.n_batches = nl;
        Ln.n_app = 0;
        Ln.n_dir = n_near;
        Ln.app_off = DBuf<int32_t>(c, nl + 1);
        BLTC_CUDA(cudaMemsetAsync(Ln.app_off.p, 0, sizeof(int32_t) * (nl + 1), s));
        Ln.app_ids = DBuf<int32_t>(c, 0);
        Ln.dir_off = std::move(near_off);
        Ln.dir_ids = std::move(near_ids);
        evaluate(c, &Ln, &tt, &ss, p, phi);
    }
    // far half: a sweep over the approximated clusters' Chebyshev grids, then interpolation
    if (nt_app > 0) {
        const int64_t npts = static_cast<int64_t>(nt_app) * P;
        require(npts < (int64_t(1) << 31), "solve_cp: too many interpolation points (clusters x (n+1)^3)");
        Tree px;
        px.ctx = c;
        px.n = npts;
        px.max_leaf = P;
        px.n_nodes = nt_app;
        px.n_leaves = nt_app;
        px.n_levels = 1;
        px.px = DBuf<double>(c, npts);
        px.py = DBuf<double>(c, npts);
        px.pz = DBuf<double>(c, npts);
        px.perm = DBuf<int32_t>(c, npts);
        px.begin = DBuf<int32_t>(c, nt_app);
        px.count = DBuf<int32_t>(c, nt_app);
        px.leaves = DBuf<int32_t>(c, nt_app);
        px.nch = DBuf<int32_t>(c, nt_app);
        px.parent = DBuf<int32_t>(c, nt_app);
        px.lo = DBuf<double>(c, 3 * static_cast<int64_t>(nt_app));
        px.hi = DBuf<double>(c, 3 * static_cast<int64_t>(nt_app));
        px.center = DBuf<double>(c, 3 * static_cast<int64_t>(nt_app));
        px.radius = DBuf<double>(c, nt_app);
        k_cp_proxy<<<nt_app, 256, 0, s>>>(tlist.p, nt_app, tt.lo.p, tt.hi.p, tt.center.p, tt.radius.p,
                                          c->cheb_table(p.degree), np1, px.px.p, px.py.p, px.pz.p, px.perm.p,
                                          px.begin.p, px.count.p, px.leaves.p, px.nch.p, px.parent.p, px.lo.p,
                                          px.hi.p, px.center.p, px.radius.p); ++c->launches;
        BLTC_LAUNCH_CHECK("cp proxy");
        Lists Lf;
        Lf.ctx = c;
        Lf.serial = c->next_serial++;
        Lf.bt = &px;
        Lf.st = &ss;
        Lf.theta = p.theta;
        Lf.degree = p.degree;
        Lf.n_batches = nt_app;
        Lf.n_app = 0;
        Lf.n_dir = n_far;
        Lf.app_off = DBuf<int32_t>(c, nt_app + 1);
        BLTC_CUDA(cudaMemsetAsync(Lf.app_off.p, 0, sizeof(int32_t) * (nt_app + 1), s));
        Lf.app_ids = DBuf<int32_t>(c, 0);
        Lf.dir_off = std::move(off_c);
        Lf.dir_ids = std::move(far_ids);
        DBuf<double> phat(c, npts);
        evaluate(c, &Lf, &px, &ss, p, phat.p);
        k_cp_l2p<<<nl, 256, sizeof(double) * P, s>>>(tt.leaves.p, tt.begin.p, tt.count.p, tt.parent.p,
                                                     tt.perm.p, tt.px.p, tt.py.p, tt.pz.p, tt.lo.p, tt.hi.p,
                                                     c->cheb_table(p.degree), tidx.p, phat.p, np1, phi); ++c->launches;
        BLTC_LAUNCH_CHECK("cp l2p");
    }
    c->mark(Context::kEnd);
}

}  // namespace bltc
