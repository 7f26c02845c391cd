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
// a sweep over the target leaves with direct lists only.  The point potentials are then
// pushed down the target tree by exact transfers and interpolated once per target.  Every
// per-target list is sorted by source batch, so sums run in a fixed order.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace bltc {
namespace {

constexpr int kThreads = 256;

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

__global__ void k_diff(const int32_t* __restrict__ off, int64_t n, int32_t* cnt) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = off[i + 1] - off[i];
}

__global__ void k_copy_last(const int32_t* off, int64_t n, int32_t* off_c, int64_t n_c) { off_c[n_c] = off[n]; }

// Each segment in ascending order, one block per segment: a bitonic sort in shared memory
// for up to 4096 entries (padded with INT_MAX), a single-thread insertion sort beyond.
constexpr int kSortMax = 4096;
__global__ void __launch_bounds__(256) k_seg_sort(const int32_t* __restrict__ off, int32_t* ids) {
    __shared__ int32_t v[kSortMax];
    const int i = blockIdx.x;
    int32_t* a = ids + off[i];
    const int m = off[i + 1] - off[i];
    if (m <= 1) return;
    if (m > kSortMax) {
        if (threadIdx.x == 0)
            for (int x = 1; x < m; ++x) {
                const int32_t key = a[x];
                int y = x - 1;
                while (y >= 0 && a[y] > key) {
                    a[y + 1] = a[y];
                    --y;
                }
                a[y + 1] = key;
            }
        return;
    }
    int n2 = 1;
    while (n2 < m) n2 <<= 1;
    for (int x = threadIdx.x; x < n2; x += blockDim.x) v[x] = x < m ? a[x] : 0x7fffffff;
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int x = threadIdx.x; x < n2; x += blockDim.x) {
                const int y = x ^ j;
                if (y > x) {
                    const bool up = (x & k) == 0;
                    const int32_t p = v[x], q = v[y];
                    if ((p > q) == up) {
                        v[x] = q;
                        v[y] = p;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int x = threadIdx.x; x < m; x += blockDim.x) a[x] = v[x];
}

// Downward pass (the transpose of the upward pass's exact transfer): a parent's interpolant
// evaluated at a child's Chebyshev points, phihat_c[k'] += sum_k L^T_k(s^c_k') phihat_T[k]
// (three (n+1)x(n+1) mode products; exact since the parent's interpolant has degree n in
// each variable).  One block per (parent, child) pair of a level; each child has one parent,
// so its row has one writer.  FP64.
__global__ void __launch_bounds__(256) k_l2l_child(const int32_t* __restrict__ nodes, const int32_t* __restrict__ nch,
                                                   const int32_t* __restrict__ child, const double* __restrict__ lo,
                                                   const double* __restrict__ hi, const double* __restrict__ cheb_t,
                                                   const int32_t* __restrict__ has, int np1, double* full) {
    extern __shared__ __align__(16) double l2l_smem[];
    const int v = nodes[blockIdx.x >> 3], ci = static_cast<int>(blockIdx.x & 7);
    if (ci >= nch[v] || !has[v]) return;
    const int c = child[8 * v + ci];
    const int n = np1 - 1, P = np1 * np1 * np1, n2 = np1 * np1;
    double* A = l2l_smem;            // the parent's values, then the second mode product
    double* Bm = A + P;
    double* Tm = Bm + P;             // [3][np1][np1], Tm_d[k][k'] = L^T_k(s^c_k')
    double* sp = Tm + 3 * n2;        // parent points [3][np1]
    const int tid = threadIdx.x;
    if (tid < 3 * np1) {
        const int d = tid / np1, k = tid - d * np1;
        sp[tid] = cheb_pt(cheb_t, k, n, lo[3 * v + d], hi[3 * v + d]);
    }
    for (int i = tid; i < P; i += blockDim.x) A[i] = full[static_cast<int64_t>(v) * P + i];
    __syncthreads();
    if (tid < 3 * np1) {
        const int d = tid / np1, kp = tid - d * np1;
        const double y = cheb_pt(cheb_t, kp, n, lo[3 * c + d], hi[3 * c + d]);
        const double* sv = sp + d * np1;
        double* col = Tm + d * n2 + kp;
        int hit = -1;
        for (int k = 0; k < np1; ++k)
            if (hit < 0 && fabs(y - sv[k]) < 2.2250738585072014e-308) hit = k;
        if (hit >= 0) {
            for (int k = 0; k < np1; ++k) col[k * np1] = k == hit ? 1.0 : 0.0;
        } else {
            double den = 0.0;
            for (int k = 0; k < np1; ++k) {
                const double w = ((k == 0 || k == n) ? 0.5 : 1.0) * ((k & 1) ? -1.0 : 1.0);
                den += w / (y - sv[k]);
            }
            for (int k = 0; k < np1; ++k) {
                const double w = ((k == 0 || k == n) ? 0.5 : 1.0) * ((k & 1) ? -1.0 : 1.0);
                col[k * np1] = (w / (y - sv[k])) / den;
            }
        }
    }
    __syncthreads();
    // B[k1',k2,k3] = sum_k1 T1[k1][k1'] A[k1,k2,k3]
    for (int i = tid; i < P; i += blockDim.x) {
        const int k1p = i / n2, r = i - k1p * n2;
        double acc = 0.0;
        for (int j = 0; j < np1; ++j) acc += Tm[j * np1 + k1p] * A[j * n2 + r];
        Bm[i] = acc;
    }
    __syncthreads();
    // C[k1',k2',k3] = sum_k2 T2[k2][k2'] B[k1',k2,k3]   (into A)
    for (int i = tid; i < P; i += blockDim.x) {
        const int k1p = i / n2, r = i - k1p * n2, k2p = r / np1, k3 = r - k2p * np1;
        double acc = 0.0;
        for (int j = 0; j < np1; ++j) acc += Tm[n2 + j * np1 + k2p] * Bm[k1p * n2 + j * np1 + k3];
        A[i] = acc;
    }
    __syncthreads();
    // child[k1',k2',k3'] += sum_k3 T3[k3][k3'] C[k1',k2',k3]
    for (int i = tid; i < P; i += blockDim.x) {
        const int k3p = i % np1, base = i - k3p;
        double acc = 0.0;
        for (int j = 0; j < np1; ++j) acc += Tm[2 * n2 + j * np1 + k3p] * A[base + j];
        full[static_cast<int64_t>(c) * P + i] += acc;
    }
}

__global__ void k_l2l_init(const int32_t* __restrict__ tidx, const double* __restrict__ phat, int64_t m,
                           int P, double* full, int32_t* has) {
    const int64_t v = blockIdx.x;
    if (v >= m) return;
    const int slot = tidx[v];
    if (threadIdx.x == 0) has[v] = slot >= 0 ? 1 : 0;
    for (int k = threadIdx.x; k < P; k += blockDim.x)
        full[v * P + k] = slot >= 0 ? phat[static_cast<int64_t>(slot) * P + k] : 0.0;
}

// has[c] |= has[parent] for the children of one level's nodes.
__global__ void k_l2l_has(const int32_t* __restrict__ nodes, int n, const int32_t* __restrict__ nch,
                          const int32_t* __restrict__ child, int32_t* has) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int v = nodes[i];
    if (!has[v]) return;
    for (int c = 0; c < nch[v]; ++c) has[child[8 * v + c]] = 1;
}

// Interpolation at the targets of each leaf from the leaf's accumulated point potentials.
__global__ void __launch_bounds__(256) k_l2p_leaf(const int32_t* __restrict__ leaves, const int32_t* __restrict__ begin,
                                                  const int32_t* __restrict__ count, const int32_t* __restrict__ perm,
                                                  const double* __restrict__ px, const double* __restrict__ py,
                                                  const double* __restrict__ pz, const double* __restrict__ lo,
                                                  const double* __restrict__ hi, const double* __restrict__ cheb_t,
                                                  const int32_t* __restrict__ has, const double* __restrict__ full,
                                                  int np1, double* phi) {
    extern __shared__ double l2p_row[];
    __shared__ double s_pts[3 * (BLTC_MAX_DEGREE + 1)];
    const int L = leaves[blockIdx.x];
    if (!has[L]) return;
    const int n = np1 - 1, P = np1 * np1 * np1;
    for (int k = threadIdx.x; k < P; k += blockDim.x) l2p_row[k] = full[static_cast<int64_t>(L) * P + k];
    if (threadIdx.x < 3 * np1) {
        const int dim = threadIdx.x / np1, k = threadIdx.x - dim * np1;
        s_pts[threadIdx.x] = cheb_pt(cheb_t, k, n, lo[3 * L + dim], hi[3 * L + dim]);
    }
    __syncthreads();
    const int tb = begin[L], nb = count[L];
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
        const double y[3] = {px[tb + t], py[tb + t], pz[tb + t]};
        double a[3][BLTC_MAX_DEGREE + 1];
        for (int dim = 0; dim < 3; ++dim) {
            const double* sv = s_pts + dim * np1;
            int hit = -1;
            for (int k = 0; k < np1; ++k)
                if (hit < 0 && fabs(y[dim] - sv[k]) < 2.2250738585072014e-308) hit = k;
            if (hit >= 0) {
                for (int k = 0; k < np1; ++k) a[dim][k] = k == hit ? 1.0 : 0.0;
            } else {
                double den = 0.0;
                for (int k = 0; k < np1; ++k) {
                    const double w = ((k == 0 || k == n) ? 0.5 : 1.0) * ((k & 1) ? -1.0 : 1.0);
                    a[dim][k] = w / (y[dim] - sv[k]);
                    den += a[dim][k];
                }
                for (int k = 0; k < np1; ++k) a[dim][k] /= den;
            }
        }
        double sum = 0.0;
        for (int k1 = 0; k1 < np1; ++k1)
            for (int k2 = 0; k2 < np1; ++k2) {
                const double a12 = a[0][k1] * a[1][k2];
                const double* row = l2p_row + (k1 * np1 + k2) * np1;
                double r3 = 0.0;
                for (int k3 = 0; k3 < np1; ++k3) r3 += a[2][k3] * row[k3];
                sum += a12 * r3;
            }
        phi[perm[tb + t]] += sum;
    }
}

}  // namespace

// Adds, for every target, the interpolant of the point potentials of the clusters holding
// it: the potentials are pushed down the target tree level by level (k_l2l_child, exact
// transfers) and each target interpolates once, from its leaf (k_l2p_leaf).
static void interpolate_down(Context* c, const Tree& tt, const int32_t* tidx, const double* phat, int degree,
                             double* phi) {
    cudaStream_t s = c->stream;
    const int np1 = degree + 1, P = np1 * np1 * np1;
    const int64_t m = tt.n_nodes;
    DBuf<double> full(c, m * P);
    DBuf<int32_t> has(c, m);
    k_l2l_init<<<static_cast<unsigned>(m), 256, 0, s>>>(tidx, phat, m, P, full.p, has.p); ++c->launches;
    // internal nodes grouped by level (host side; the tree has few nodes per particle)
    std::vector<int32_t> lev(static_cast<size_t>(m)), nch(static_cast<size_t>(m));
    BLTC_CUDA(cudaMemcpyAsync(lev.data(), tt.level.p, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
    BLTC_CUDA(cudaMemcpyAsync(nch.data(), tt.nch.p, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s));
    BLTC_CUDA(cudaStreamSynchronize(s));
    const int nlv = std::max(tt.n_levels, 1);
    std::vector<int32_t> off(static_cast<size_t>(nlv) + 1, 0), order;
    order.reserve(static_cast<size_t>(m));
    for (int L = 0; L < nlv; ++L) {
        for (int64_t v = 0; v < m; ++v)
            if (lev[static_cast<size_t>(v)] == L && nch[static_cast<size_t>(v)] > 0) order.push_back(static_cast<int32_t>(v));
        off[static_cast<size_t>(L) + 1] = static_cast<int32_t>(order.size());
    }
    DBuf<int32_t> nodes(c, std::max<int64_t>(static_cast<int64_t>(order.size()), 1));
    if (!order.empty())
        BLTC_CUDA(cudaMemcpyAsync(nodes.p, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice, s));
    const size_t smem = sizeof(double) * (2 * static_cast<size_t>(P) + 3 * static_cast<size_t>(np1) * np1 + 3 * np1);
    const int kmax = BLTC_MAX_DEGREE + 1;
    BLTC_CUDA(cudaFuncSetAttribute(k_l2l_child, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   static_cast<int>(sizeof(double) * (2 * kmax * kmax * kmax + 3 * kmax * kmax + 3 * kmax))));
    const double* cheb = c->cheb_table(degree);
    for (int L = 0; L < nlv; ++L) {
        const int n = off[static_cast<size_t>(L) + 1] - off[static_cast<size_t>(L)];
        if (n == 0) continue;
        const int32_t* lv = nodes.p + off[static_cast<size_t>(L)];
        k_l2l_child<<<8 * n, 256, smem, s>>>(lv, tt.nch.p, tt.child.p, tt.lo.p, tt.hi.p, cheb, has.p, np1, full.p); ++c->launches;
        k_l2l_has<<<grid_for(n, 256), 256, 0, s>>>(lv, n, tt.nch.p, tt.child.p, has.p); ++c->launches;
    }
    BLTC_LAUNCH_CHECK("l2l");
    k_l2p_leaf<<<static_cast<unsigned>(tt.n_leaves), 256, sizeof(double) * P, s>>>(
        tt.leaves.p, tt.begin.p, tt.count.p, tt.perm.p, tt.px.p, tt.py.p, tt.pz.p, tt.lo.p, tt.hi.p, cheb, has.p,
        full.p, np1, phi); ++c->launches;
    BLTC_LAUNCH_CHECK("l2p");
    BLTC_CUDA(cudaStreamSynchronize(s));        // `order` lives on the host stack
}

// The synthetic batch tree whose leaves are the Chebyshev grids of the target clusters
// tlist[0..nt_app) (P points each, identity permutation).
static void make_proxy_tree(Context* c, const Tree& tt, const int32_t* tlist, int32_t nt_app, int degree,
                            Tree* px) {
    const int np1 = degree + 1, P = np1 * np1 * np1;
    const int64_t npts = static_cast<int64_t>(nt_app) * P;
    px->ctx = c;
    px->n = npts;
    px->max_leaf = P;
    px->n_nodes = nt_app;
    px->n_leaves = nt_app;
    px->n_levels = 1;
    px->px = DBuf<double>(c, npts);
    px->py = DBuf<double>(c, npts);
    px->pz = DBuf<double>(c, npts);
    px->perm = DBuf<int32_t>(c, npts);
    px->begin = DBuf<int32_t>(c, nt_app);
    px->count = DBuf<int32_t>(c, nt_app);
    px->leaves = DBuf<int32_t>(c, nt_app);
    px->nch = DBuf<int32_t>(c, nt_app);
    px->parent = DBuf<int32_t>(c, nt_app);
    px->lo = DBuf<double>(c, 3 * static_cast<int64_t>(nt_app));
    px->hi = DBuf<double>(c, 3 * static_cast<int64_t>(nt_app));
    px->center = DBuf<double>(c, 3 * static_cast<int64_t>(nt_app));
    px->radius = DBuf<double>(c, nt_app);
    k_cp_proxy<<<nt_app, 256, 0, c->stream>>>(tlist, nt_app, tt.lo.p, tt.hi.p, tt.center.p, tt.radius.p,
                                              c->cheb_table(degree), np1, px->px.p, px->py.p, px->pz.p,
                                              px->perm.p, px->begin.p, px->count.p, px->leaves.p, px->nch.p,
                                              px->parent.p, px->lo.p, px->hi.p, px->center.p, px->radius.p); ++c->launches;
    BLTC_LAUNCH_CHECK("proxy tree");
}

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
    k_seg_sort<<<static_cast<unsigned>(m), 256, 0, s>>>(far_off.p, far_ids.p); ++c->launches;
    k_seg_sort<<<static_cast<unsigned>(nl), 256, 0, s>>>(near_off.p, near_ids.p); ++c->launches;
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
        make_proxy_tree(c, tt, tlist.p, nt_app, p.degree, &px);
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
        interpolate_down(c, tt, tidx.p, phat.p, p.degree, phi);
    }
    c->mark(Context::kEnd);
}

}  // namespace bltc

// ---- the cluster-cluster variant (dual tree traversal, future work of Sec. V) -----------
//
// Reading (the paper names the variant without defining it): DualTraversal(T, S) from the
// two roots; if (r_T + r_S)/R < theta the pair interacts as CC (P < N_T and P < N_S: point
// potentials of T from the modified charges of S), CP (P < N_T only: point potentials of T
// from S's particles), PC (P < N_S only: T's targets from S's modified charges) or PP (both
// exact); otherwise leaf-leaf pairs are PP and else the larger cluster is split (T when S is
// a leaf or r_T >= r_S and T is not a leaf).  The traversal runs level by level on the GPU:
// each level's pairs are classified, their children pairs and interactions counted, scanned
// and written in frontier order, so the lists are deterministic.  Then, as for the
// cluster-particle variant, CC and CP terms become a sweep over the target clusters'
// Chebyshev grids (approximation entries = CC sources, direct entries = CP sources), PC and
// PP terms a sweep over the target leaves, and interpolate_down interpolates.

namespace bltc {
namespace {

struct DualArgs {
    const int32_t *t_nch, *t_child, *t_count;
    const double *t_center, *t_radius;
    const int32_t *s_nch, *s_child, *s_count;
    const double *s_center, *s_radius;
    double theta;
    int64_t P;
};

enum { kCC = 0, kCP = 1, kPC = 2, kPP = 3, kSplitT = 4, kSplitS = 5 };

// One frontier pair's decision: Eq. 13's geometric test, then the size tests, then the split rule
// of the dual traversal (FP64 with explicit rounding, evaluated left to right).
__device__ __forceinline__ int dual_decide(const DualArgs& a, int T, int S) {
    const double dx = __dsub_rn(a.t_center[3 * T], a.s_center[3 * S]);
    const double dy = __dsub_rn(a.t_center[3 * T + 1], a.s_center[3 * S + 1]);
    const double dz = __dsub_rn(a.t_center[3 * T + 2], a.s_center[3 * S + 2]);
    const double R = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
    const double ratio = __ddiv_rn(__dadd_rn(a.t_radius[T], a.s_radius[S]), R);
    const bool t_leaf = a.t_nch[T] == 0, s_leaf = a.s_nch[S] == 0;
    if (ratio < a.theta) {
        const bool tc = a.P < a.t_count[T], sc = a.P < a.s_count[S];
        return tc ? (sc ? kCC : kCP) : (sc ? kPC : kPP);
    }
    if (t_leaf && s_leaf) return kPP;
    if (s_leaf || (!t_leaf && a.t_radius[T] >= a.s_radius[S])) return kSplitT;
    return kSplitS;
}

// Pass 0: per pair, its children count and one flag per interaction kind.
// Pass 1: write the children into the next frontier and the pair into its kind's list.
template <bool kFill>
__global__ void k_dual_level(DualArgs a, const int2* __restrict__ fr, int64_t n, int32_t* nchild,
                             int32_t* kflag, const int32_t* __restrict__ child_off,
                             const int32_t* __restrict__ kind_off, const int32_t* __restrict__ base,
                             int2* next, int2* lists) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int T = fr[i].x, S = fr[i].y;
    const int d = dual_decide(a, T, S);
    if (!kFill) {
        nchild[i] = d == kSplitT ? a.t_nch[T] : (d == kSplitS ? a.s_nch[S] : 0);
        for (int k = 0; k < 4; ++k) kflag[k * n + i] = d == k ? 1 : 0;
        return;
    }
    if (d == kSplitT) {
        for (int c = 0; c < a.t_nch[T]; ++c) next[child_off[i] + c] = make_int2(a.t_child[8 * T + c], S);
    } else if (d == kSplitS) {
        for (int c = 0; c < a.s_nch[S]; ++c) next[child_off[i] + c] = make_int2(T, a.s_child[8 * S + c]);
    } else {
        lists[base[d] + kind_off[d * n + i]] = make_int2(T, S);
    }
}

// Per target node (or per target leaf, expanding each node to its leaves): count, then fill
// the source ids of a pair list.
template <bool kFill>
__global__ void k_pairs_to_targets(const int2* __restrict__ pairs, int64_t n, bool to_leaves,
                                   const int32_t* __restrict__ t_begin, const int32_t* __restrict__ t_count,
                                   const int32_t* __restrict__ leaf_begin, int n_leaves, int32_t* cnt,
                                   const int32_t* __restrict__ off, int32_t* ids) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int T = pairs[e].x, S = pairs[e].y;
    if (!to_leaves) {
        const int pos = atomicAdd(&cnt[T], 1);
        if (kFill) ids[off[T] + pos] = S;
        return;
    }
    int i0, i1;
    leaf_range(leaf_begin, n_leaves, t_begin[T], t_begin[T] + t_count[T], &i0, &i1);
    for (int i = i0; i < i1; ++i) {
        const int pos = atomicAdd(&cnt[i], 1);
        if (kFill) ids[off[i] + pos] = S;
    }
}

__global__ void k_or_nonzero(const int32_t* a, const int32_t* b, int64_t n, int32_t* flag) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = (a[i] > 0 || b[i] > 0) ? 1 : 0;
}

// Compacted offsets of both lists for the flagged target nodes.
__global__ void k_cc_compact(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                             const int32_t* __restrict__ offA, const int32_t* __restrict__ offD,
                             int64_t m, int32_t* tlist, int32_t* tidx, int32_t* offA_c, int32_t* offD_c) {
    const int64_t T = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (T >= m) return;
    if (flag[T]) {
        const int p = pos[T];
        tlist[p] = static_cast<int32_t>(T);
        tidx[T] = p;
        offA_c[p] = offA[T];
        offD_c[p] = offD[T];
    } else {
        tidx[T] = -1;
    }
}

}  // namespace

namespace {

// CSR (over n_keys targets) of the source ids of a pair list, each segment in ascending
// source id.  Returns the number of entries.
int64_t pairs_csr(Context* c, const int2* pairs, int64_t n, bool to_leaves, const Tree& tt,
                  const int32_t* leaf_begin, int64_t n_keys, DBuf<int32_t>* off, DBuf<int32_t>* ids) {
    cudaStream_t s = c->stream;
    DBuf<int32_t> cnt(c, n_keys), tot(c, 2);
    *off = DBuf<int32_t>(c, n_keys + 1);
    BLTC_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * n_keys, s));
    const int nl = static_cast<int>(tt.n_leaves);
    if (n > 0) {
        k_pairs_to_targets<false><<<grid_for(n, kThreads), kThreads, 0, s>>>(
            pairs, n, to_leaves, tt.begin.p, tt.count.p, leaf_begin, nl, cnt.p, nullptr, nullptr); ++c->launches;
    }
    exclusive_scan_i32(c, cnt.p, off->p, n_keys, tot.p);
    k_cp_total<<<1, 1, 0, s>>>(off->p, n_keys, tot.p); ++c->launches;
    const int32_t total = *reinterpret_cast<const int32_t*>(c->read_words(tot.p, 1));
    *ids = DBuf<int32_t>(c, total);
    BLTC_CUDA(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * n_keys, s));
    if (n > 0) {
        k_pairs_to_targets<true><<<grid_for(n, kThreads), kThreads, 0, s>>>(
            pairs, n, to_leaves, tt.begin.p, tt.count.p, leaf_begin, nl, cnt.p, off->p, ids->p); ++c->launches;
    }
    k_seg_sort<<<static_cast<unsigned>(n_keys), 256, 0, s>>>(off->p, ids->p); ++c->launches;
    BLTC_LAUNCH_CHECK("pairs csr");
    return total;
}

}  // namespace

void dual_lists(Context* c, const Tree& tt, const Tree& st, double theta, int degree,
                DBuf<int2> (&lists)[4], int64_t (&counts)[4]) {
    require(degree >= 1 && degree <= BLTC_MAX_DEGREE, "dual lists: degree out of range");
    cudaStream_t s = c->stream;
    DualArgs a{tt.nch.p, tt.child.p, tt.count.p, tt.center.p, tt.radius.p,
               st.nch.p, st.child.p, st.count.p, st.center.p, st.radius.p,
               theta, static_cast<int64_t>(degree + 1) * (degree + 1) * (degree + 1)};
    std::vector<DBuf<int2>> parts[4];
    std::vector<int64_t> part_n[4];
    DBuf<int2> fr(c, 1);
    const int2 root = make_int2(0, 0);
    BLTC_CUDA(cudaMemcpyAsync(fr.p, &root, sizeof(int2), cudaMemcpyHostToDevice, s));
    int64_t n = 1;
    DBuf<int32_t> tot(c, 6);
    while (n > 0) {
        DBuf<int32_t> nchild(c, n), kflag(c, 4 * n), child_off(c, n), kind_off(c, 4 * n), base(c, 4);
        k_dual_level<false><<<grid_for(n, kThreads), kThreads, 0, s>>>(a, fr.p, n, nchild.p, kflag.p, nullptr,
                                                                    nullptr, nullptr, nullptr, nullptr); ++c->launches;
        exclusive_scan_i32(c, nchild.p, child_off.p, n, tot.p);
        for (int k = 0; k < 4; ++k) exclusive_scan_i32(c, kflag.p + k * n, kind_off.p + k * n, n, tot.p + 1 + k);
        BLTC_LAUNCH_CHECK("dual count");
        const int32_t* w = reinterpret_cast<const int32_t*>(c->read_words(tot.p, 3));
        const int64_t n_next = w[0];
        int64_t nk[4];
        for (int k = 0; k < 4; ++k) nk[k] = w[1 + k];
        DBuf<int2> next(c, std::max<int64_t>(n_next, 1));
        // this level's interactions go to fresh arrays, concatenated at the end
        DBuf<int2> lev(c, std::max<int64_t>(nk[0] + nk[1] + nk[2] + nk[3], 1));
        const int32_t hbase[4] = {0, static_cast<int32_t>(nk[0]), static_cast<int32_t>(nk[0] + nk[1]),
                                  static_cast<int32_t>(nk[0] + nk[1] + nk[2])};
        BLTC_CUDA(cudaMemcpyAsync(base.p, hbase, sizeof(hbase), cudaMemcpyHostToDevice, s));
        k_dual_level<true><<<grid_for(n, kThreads), kThreads, 0, s>>>(a, fr.p, n, nullptr, nullptr, child_off.p,
                                                                   kind_off.p, base.p, next.p, lev.p); ++c->launches;
        BLTC_LAUNCH_CHECK("dual fill");
        BLTC_CUDA(cudaStreamSynchronize(s));          // hbase is on the host stack
        for (int k = 0; k < 4; ++k) {
            if (nk[k] == 0) continue;
            DBuf<int2> part(c, nk[k]);
            BLTC_CUDA(cudaMemcpyAsync(part.p, lev.p + hbase[k], sizeof(int2) * nk[k], cudaMemcpyDeviceToDevice, s));
            parts[k].push_back(std::move(part));
            part_n[k].push_back(nk[k]);
        }
        fr = std::move(next);
        n = n_next;
    }
    for (int k = 0; k < 4; ++k) {
        int64_t total = 0;
        for (int64_t v : part_n[k]) total += v;
        counts[k] = total;
        lists[k] = DBuf<int2>(c, std::max<int64_t>(total, 1));
        int64_t o = 0;
        for (size_t i = 0; i < parts[k].size(); ++i) {
            BLTC_CUDA(cudaMemcpyAsync(lists[k].p + o, parts[k][i].p, sizeof(int2) * part_n[k][i],
                                      cudaMemcpyDeviceToDevice, s));
            o += part_n[k][i];
        }
    }
}

void solve_device_cc(Context* c, const double* tx, const double* ty, const double* tz, int64_t nt,
                     const double* sx, const double* sy, const double* sz, const double* sq, int64_t ns,
                     const bltc_params& p, double* phi) {
    cudaStream_t s = c->stream;
    const int np1 = p.degree + 1, P = np1 * np1 * np1;
    c->mark(Context::kStart);
    Tree ts, st;
    build_tree(c, sx, sy, sz, sq, ns, p.leaf_size, &st);            // source clusters
    const bool same = tx == sx && ty == sy && tz == sz && nt == ns && p.leaf_size == p.batch_size;
    if (!same) build_tree(c, tx, ty, tz, nullptr, nt, p.batch_size, &ts);   // target clusters
    Tree& tt = same ? st : ts;
    c->mark(Context::kTrees);
    DBuf<int2> lists[4];
    int64_t cnt[4];
    dual_lists(c, tt, st, p.theta, p.degree, lists, cnt);
    c->mark(Context::kLists);
    compute_modified_charges(c, &st, nullptr, p.degree, p.precision);   // every cluster with N > P
    c->mark(Context::kUpward);

    const int64_t m = tt.n_nodes;
    const int nl = static_cast<int>(tt.n_leaves);
    DBuf<int32_t> leaf_begin(c, nl);
    k_leaf_begin<<<grid_for(nl, kThreads), kThreads, 0, s>>>(tt.leaves.p, tt.begin.p, nl, leaf_begin.p); ++c->launches;
    // PC and PP: per target leaf, then a sweep over the target leaves
    {
        DBuf<int32_t> offA, idsA, offD, idsD;
        const int64_t na = pairs_csr(c, lists[kPC].p, cnt[kPC], true, tt, leaf_begin.p, nl, &offA, &idsA);
        const int64_t nd = pairs_csr(c, lists[kPP].p, cnt[kPP], true, tt, leaf_begin.p, nl, &offD, &idsD);
        Lists Ln;
        Ln.ctx = c;
        Ln.serial = c->next_serial++;
        Ln.bt = &tt;
        Ln.st = &st;
        Ln.theta = p.theta;
        Ln.degree = p.degree;
        Ln.n_batches = nl;
        Ln.n_app = na;
        Ln.n_dir = nd;
        Ln.app_off = std::move(offA);
        Ln.app_ids = std::move(idsA);
        Ln.dir_off = std::move(offD);
        Ln.dir_ids = std::move(idsD);
        evaluate(c, &Ln, &tt, &st, p, phi);
    }
    // CC and CP: per target node, a sweep over the approximated clusters' Chebyshev grids
    DBuf<int32_t> offA, idsA, offD, idsD;
    const int64_t na = pairs_csr(c, lists[kCC].p, cnt[kCC], false, tt, leaf_begin.p, m, &offA, &idsA);
    const int64_t nd = pairs_csr(c, lists[kCP].p, cnt[kCP], false, tt, leaf_begin.p, m, &offD, &idsD);
    if (na + nd > 0) {
        DBuf<int32_t> cntA(c, m), cntD(c, m), flag(c, m), pos(c, m), tidx(c, m), tot(c, 2);
        // per-node counts from the offsets
        k_diff<<<grid_for(m, kThreads), kThreads, 0, s>>>(offA.p, m, cntA.p); ++c->launches;
        k_diff<<<grid_for(m, kThreads), kThreads, 0, s>>>(offD.p, m, cntD.p); ++c->launches;
        k_or_nonzero<<<grid_for(m, kThreads), kThreads, 0, s>>>(cntA.p, cntD.p, m, flag.p); ++c->launches;
        exclusive_scan_i32(c, flag.p, pos.p, m, tot.p);
        const int32_t nt_app = *reinterpret_cast<const int32_t*>(c->read_words(tot.p, 1));
        DBuf<int32_t> tlist(c, nt_app), offA_c(c, nt_app + 1), offD_c(c, nt_app + 1);
        k_cc_compact<<<grid_for(m, kThreads), kThreads, 0, s>>>(flag.p, pos.p, offA.p, offD.p, m, tlist.p, tidx.p,
                                                             offA_c.p, offD_c.p); ++c->launches;
        k_copy_last<<<1, 1, 0, s>>>(offA.p, m, offA_c.p, nt_app); ++c->launches;
        k_copy_last<<<1, 1, 0, s>>>(offD.p, m, offD_c.p, nt_app); ++c->launches;
        BLTC_LAUNCH_CHECK("cc compact");
        const int64_t npts = static_cast<int64_t>(nt_app) * P;
        require(npts < (int64_t(1) << 31), "solve_cc: too many interpolation points (clusters x (n+1)^3)");
        Tree px;
        make_proxy_tree(c, tt, tlist.p, nt_app, p.degree, &px);
        Lists Lf;
        Lf.ctx = c;
        Lf.serial = c->next_serial++;
        Lf.bt = &px;
        Lf.st = &st;
        Lf.theta = p.theta;
        Lf.degree = p.degree;
        Lf.n_batches = nt_app;
        Lf.n_app = na;
        Lf.n_dir = nd;
        Lf.app_off = std::move(offA_c);
        Lf.app_ids = std::move(idsA);
        Lf.dir_off = std::move(offD_c);
        Lf.dir_ids = std::move(idsD);
        DBuf<double> phat(c, npts);
        evaluate(c, &Lf, &px, &st, p, phat.p);
        interpolate_down(c, tt, tidx.p, phat.p, p.degree, phi);
    }
    c->mark(Context::kEnd);
}

}  // namespace bltc
