// upward.cu -- A2: modified charges of the source clusters (Eq. 12, Sec. II-C).
//
//   qhat_k = sum_{y_j in C} L_k1(y_j1) L_k2(y_j2) L_k3(y_j3) q_j,   k = (k1, k2, k3)
//
// with L_k(y) = (w_k / (y - s_k)) / sum_k' (w_k' / (y - s_k')) on the Chebyshev points of
// the second kind of C's box (Eq. 4, 6, 7), and L_k(y) = delta_{k k'} enforced when y is
// within DBL_MIN of s_k' (Sec. II-C).  The factorisation of Eq. 14-15 (one pass per
// particle for the three 1D denominators, then a contraction over the particles) maps to:
//   item = (cluster, chunk of <= 2048 particles), one block per item;
//   phase A: one thread per (particle, dimension) computes the n+1 one-dimensional factors
//            in FP64 (differences y - s_k, exact-hit test; FP32 after the difference in
//            the mixed path) and folds q_j into the first dimension;
//   phase B: one thread per (k1, k2) pair (times particle groups) accumulates
//            sum_j a1[k1] a2[k2] a3[k3] over the chunk for all k3 in registers;
//   a second kernel sums the chunk partials of a cluster in chunk order (FP64).
// Only clusters that some batch approximates need modified charges (a cluster's charges
// do not depend on which batches use it).
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace bltc {
namespace {

constexpr int kThreads = 512;
constexpr int kTile = 128;            // particles per phase-A tile
constexpr int kItem = 2048;           // particles per item
constexpr int kMaxNp1 = BLTC_MAX_DEGREE + 1;

struct UpArgs {
    const double *px, *py, *pz, *pq;
    const int32_t* begin;
    const int32_t* count;
    const double* lo;
    const double* hi;
    const double* cheb_t;
    const int32_t* slot_node;         // slot -> node
    const int4* items;                // {slot, first particle, end particle, -}
    double* partial;                  // [n_items * P]
    int np1;
};

// Chebyshev point k of [lo, hi] (Eq. 6 mapped linearly; s_0 = hi and s_n = lo exactly).
__device__ __forceinline__ double cheb_point(const double* t, int k, int n, double lo, double hi) {
    if (k == 0) return hi;
    if (k == n) return lo;
    return __dadd_rn(lo, __dmul_rn(__dmul_rn(0.5, __dadd_rn(t[k], 1.0)), __dsub_rn(hi, lo)));
}

template <typename F>
__global__ void __launch_bounds__(kThreads) k_upward_partial(UpArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F* fac = reinterpret_cast<F*>(smem_raw);       // [3][np1][kTile + 1]
    const int np1 = a.np1, n = np1 - 1;
    const int pairs = np1 * np1;
    const int P = pairs * np1;
    const int G = max(1, kThreads / pairs);
    const int stride = kTile + 1;
    const int4 it = a.items[blockIdx.x];
    const int node = a.slot_node[it.x];
    const double lo[3] = {a.lo[3 * node], a.lo[3 * node + 1], a.lo[3 * node + 2]};
    const double hi[3] = {a.hi[3 * node], a.hi[3 * node + 1], a.hi[3 * node + 2]};
    const int tid = threadIdx.x;
    const bool active = tid < pairs * G;
    const int p = tid % pairs, g = tid / pairs;
    const int k1 = p / np1, k2 = p % np1;
    // Per-thread sums over its particles: blocks of the tile summed in F, folded into a
    // TwoSum (hi, lo) accumulator so FP32 rounding does not grow with the particle count.
    F acc[kMaxNp1], lo_acc[kMaxNp1];
#pragma unroll
    for (int k = 0; k < kMaxNp1; ++k) acc[k] = lo_acc[k] = F(0);
    // the 3(n+1) Chebyshev points of this cluster, once per block
    __shared__ double s_pts[3 * kMaxNp1];
    if (tid < 3 * np1) {
        const int d = tid / np1, k = tid - d * np1;
        s_pts[tid] = cheb_point(a.cheb_t, k, n, d == 0 ? lo[0] : (d == 1 ? lo[1] : lo[2]),
                                d == 0 ? hi[0] : (d == 1 ? hi[1] : hi[2]));
    }

    for (int j0 = it.y; j0 < it.z; j0 += kTile) {
        const int m = min(kTile, it.z - j0);
        __syncthreads();
        if (tid < 3 * kTile) {
            const int j = tid % kTile, d = tid / kTile;
            if (j < m) {
                const int pos = j0 + j;
                const double yv = d == 0 ? a.px[pos] : (d == 1 ? a.py[pos] : a.pz[pos]);
                const double* pts = s_pts + d * np1;
                const double qv = d == 0 ? a.pq[pos] : 1.0;
                double dk[kMaxNp1];
                int hit = -1;
#pragma unroll
                for (int k = 0; k < kMaxNp1; ++k) {
                    if (k < np1) {
                        dk[k] = yv - pts[k];
                        // FP64: |y - s_k| < DBL_MIN.  Mixed: the FP32 difference underflows
                        // (|fp32(y - s_k)| < FLT_MIN), a superset changing L by < 1e-29.
                        const bool h = sizeof(F) == 4
                                           ? fabsf(__double2float_rn(dk[k])) < 1.17549435e-38f
                                           : fabs(dk[k]) < 2.2250738585072014e-308;
                        if (h && hit < 0) hit = k;
                    }
                }
                F* row = fac + d * np1 * stride + j;
                if (hit >= 0) {
#pragma unroll
                    for (int k = 0; k < kMaxNp1; ++k)
                        if (k < np1) row[k * stride] = k == hit ? F(qv) : F(0);
                } else {
                    F raw[kMaxNp1];
                    F den = F(0), den_lo = F(0);
#pragma unroll
                    for (int k = 0; k < kMaxNp1; ++k) {
                        if (k < np1) {
                            const F w = ((k == 0 || k == n) ? F(0.5) : F(1)) * ((k & 1) ? F(-1) : F(1));
                            raw[k] = w / F(dk[k]);
                            if (sizeof(F) == 4) {
                                // the barycentric denominator by TwoSum: its terms alternate
                                // in sign, and a plain FP32 sum loses digits to cancellation
                                const F s = den + raw[k];
                                const F bb = s - den;
                                den_lo += (den - (s - bb)) + (raw[k] - bb);
                                den = s;
                            } else {
                                den += raw[k];
                            }
                        }
                    }
                    const F scale = F(qv) / (den + den_lo);
#pragma unroll
                    for (int k = 0; k < kMaxNp1; ++k)
                        if (k < np1) row[k * stride] = raw[k] * scale;
                }
            }
        }
        __syncthreads();
        if (active) {
            const F* f0 = fac + k1 * stride;
            const F* f1 = fac + (np1 + k2) * stride;
            const F* f2 = fac + 2 * np1 * stride;
            if constexpr (sizeof(F) == 4) {
                F blk[kMaxNp1];
#pragma unroll
                for (int k = 0; k < kMaxNp1; ++k) blk[k] = F(0);
                for (int j = g; j < m; j += G) {
                    const F a12 = f0[j] * f1[j];
#pragma unroll
                    for (int k = 0; k < kMaxNp1; ++k)
                        if (k < np1) blk[k] += a12 * f2[k * stride + j];
                }
#pragma unroll
                for (int k = 0; k < kMaxNp1; ++k) {
                    if (k < np1) {
                        const F s = acc[k] + blk[k];
                        const F bb = s - acc[k];
                        lo_acc[k] += (acc[k] - (s - bb)) + (blk[k] - bb);
                        acc[k] = s;
                    }
                }
            } else {
                for (int j = g; j < m; j += G) {
                    const F a12 = f0[j] * f1[j];
#pragma unroll
                    for (int k = 0; k < kMaxNp1; ++k)
                        if (k < np1) acc[k] += a12 * f2[k * stride + j];
                }
            }
        }
    }
    // Sum the particle groups in a fixed order.
    __syncthreads();
    F* red = fac;                                   // [G][P]
    if (active) {
#pragma unroll
        for (int k = 0; k < kMaxNp1; ++k)
            if (k < np1) red[g * P + p * np1 + k] = acc[k] + lo_acc[k];
    }
    __syncthreads();
    double* out = a.partial + static_cast<int64_t>(blockIdx.x) * P;
    for (int o = tid; o < P; o += kThreads) {
        double s = 0.0;
        for (int gg = 0; gg < G; ++gg) s += static_cast<double>(red[gg * P + o]);
        out[o] = s;
    }
}

__global__ void k_upward_reduce(const double* __restrict__ partial,
                                const int32_t* __restrict__ item0, int P, double* qhat64,
                                float* qhat32) {
    const int slot = blockIdx.x;
    const int i0 = item0[slot], i1 = item0[slot + 1];
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        double s = 0.0;
        for (int i = i0; i < i1; ++i) s += partial[static_cast<int64_t>(i) * P + k];
        qhat64[static_cast<int64_t>(slot) * P + k] = s;
        if (qhat32) qhat32[static_cast<int64_t>(slot) * P + k] = static_cast<float>(s);
    }
}

__global__ void k_mark_from_lists(const int32_t* __restrict__ app_ids, int64_t n,
                                  int32_t* flag) {
    int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) flag[app_ids[i]] = 1;
}

__global__ void k_mark_by_size(const int32_t* __restrict__ count, int64_t m, int64_t P,
                               int32_t* flag) {
    int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < m) flag[v] = static_cast<int64_t>(count[v]) > P ? 1 : 0;
}

__global__ void k_slots(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                        const int32_t* __restrict__ count, const int32_t* __restrict__ nch,
                        int64_t m, int32_t* qslot, int32_t* slot_node, int32_t* slot_items) {
    int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= m) return;
    if (flag[v]) {
        qslot[v] = pos[v];
        slot_node[pos[v]] = static_cast<int32_t>(v);
        // particles are summed only at the leaves; parents come from their children (M2M)
        slot_items[pos[v]] = nch[v] == 0 ? (count[v] + kItem - 1) / kItem : 0;
    } else {
        qslot[v] = -1;
    }
}

__global__ void k_items(const int32_t* __restrict__ slot_node,
                        const int32_t* __restrict__ item0, const int32_t* __restrict__ begin,
                        const int32_t* __restrict__ count, int64_t n_slots, int4* items) {
    int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= n_slots) return;
    const int v = slot_node[s];
    const int b = begin[v], c = count[v];
    // a slot owns items item0[s] .. item0[s+1]-1: none for internal nodes (built by M2M)
    const int i1 = item0[s + 1];
    for (int i = item0[s], p0 = b; i < i1; ++i, p0 += kItem)
        items[i] = make_int4(static_cast<int>(s), p0, min(b + c, p0 + kItem), 0);
}

__global__ void k_append_total(int32_t* off, int64_t n, const int32_t* total) { off[n] = *total; }

// Clusters whose modified charges the M2M pass needs: the marked ones and, level by level,
// every descendant of a marked one (a parent's charges are built from all of its children).
__global__ void k_propagate(const int32_t* __restrict__ level, const int32_t* __restrict__ parent,
                            int64_t m, int L, int32_t* flag) {
    int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < m && level[v] == L && flag[parent[v]]) flag[v] = 1;
}

// Marked internal nodes grouped by level (order within a level is irrelevant).
__global__ void k_level_hist(const int32_t* __restrict__ flag, const int32_t* __restrict__ nch,
                             const int32_t* __restrict__ level, int64_t m, int32_t* hist) {
    int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < m && flag[v] && nch[v] > 0) atomicAdd(&hist[level[v]], 1);
}

__global__ void k_level_fill(const int32_t* __restrict__ flag, const int32_t* __restrict__ nch,
                             const int32_t* __restrict__ level, int64_t m,
                             const int32_t* __restrict__ level_off, int32_t* cursor, int32_t* list) {
    int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v < m && flag[v] && nch[v] > 0) {
        const int L = level[v];
        list[level_off[L] + atomicAdd(&cursor[L], 1)] = static_cast<int32_t>(v);
    }
}

struct M2MArgs {
    const int32_t* nch;
    const int32_t* child;
    const int32_t* qslot;
    const double* lo;
    const double* hi;
    const double* cheb_t;
    double* qhat64;
    float* qhat32;
    int np1;
};

// Exact transfer of the children's modified charges to their parent (NEXT to Eq. 12: the
// parent's Lagrange polynomials L^P_k have degree n in each variable, so a child's tensor
// interpolant reproduces them exactly and
//   qhat^P_k = sum_children sum_k' L^P_k1(s^c_k'1) L^P_k2(s^c_k'2) L^P_k3(s^c_k'3) qhat^c_k').
// One block per parent: for each child, the three (n+1)x(n+1) matrices T_l[k][k'] =
// L^P_k(s^c_k'l) (barycentric form, exact hits as in Sec. II-C), then three mode products.
// FP64 throughout.
__global__ void __launch_bounds__(256) k_m2m(M2MArgs a, const int32_t* __restrict__ nodes) {
    extern __shared__ __align__(16) double m2m_smem[];
    const int v = nodes[blockIdx.x];
    const int np1 = a.np1, n = np1 - 1, P = np1 * np1 * np1, n2 = np1 * np1;
    double* A = m2m_smem;            // child charges, then the second mode product
    double* Bm = A + P;              // first mode product
    double* out = Bm + P;            // the parent's charges
    double* T = out + P;             // [3][np1][np1]
    double* sp = T + 3 * n2;         // parent points [3][np1]
    const int tid = threadIdx.x;
    if (tid < 3 * np1) {
        const int d = tid / np1, k = tid - d * np1;
        sp[tid] = cheb_point(a.cheb_t, k, n, a.lo[3 * v + d], a.hi[3 * v + d]);
    }
    for (int i = tid; i < P; i += blockDim.x) out[i] = 0.0;
    const int nc = a.nch[v];
    for (int ci = 0; ci < nc; ++ci) {
        const int c = a.child[8 * v + ci];
        __syncthreads();
        const double* qc = a.qhat64 + static_cast<int64_t>(a.qslot[c]) * P;
        for (int i = tid; i < P; i += blockDim.x) A[i] = qc[i];
        if (tid < 3 * np1) {
            // column k' of T_d: the parent's 1-D Lagrange values at the child's point s^c_k'
            const int d = tid / np1, kp = tid - d * np1;
            const double y = cheb_point(a.cheb_t, kp, n, a.lo[3 * c + d], a.hi[3 * c + d]);
            const double* s = sp + d * np1;
            double* col = T + d * n2 + kp;            // T_d[k][kp] at col[k * np1]
            int hit = -1;
            for (int k = 0; k < np1; ++k)
                if (hit < 0 && fabs(y - s[k]) < 2.2250738585072014e-308) hit = k;
            if (hit >= 0) {
                for (int k = 0; k < np1; ++k) col[k * np1] = k == hit ? 1.0 : 0.0;
            } else {
                double den = 0.0;
                for (int k = 0; k < np1; ++k) {
                    const double w = ((k == 0 || k == n) ? 0.5 : 1.0) * ((k & 1) ? -1.0 : 1.0);
                    den += w / (y - s[k]);
                }
                for (int k = 0; k < np1; ++k) {
                    const double w = ((k == 0 || k == n) ? 0.5 : 1.0) * ((k & 1) ? -1.0 : 1.0);
                    col[k * np1] = (w / (y - s[k])) / den;
                }
            }
        }
        __syncthreads();
        // B[k1,k2',k3'] = sum_k1' T1[k1][k1'] A[k1',k2',k3']
        for (int i = tid; i < P; i += blockDim.x) {
            const int k1 = i / n2, r = i - k1 * n2;
            double acc = 0.0;
            for (int j = 0; j < np1; ++j) acc += T[k1 * np1 + j] * A[j * n2 + r];
            Bm[i] = acc;
        }
        __syncthreads();
        // C[k1,k2,k3'] = sum_k2' T2[k2][k2'] B[k1,k2',k3']   (into A)
        for (int i = tid; i < P; i += blockDim.x) {
            const int k1 = i / n2, r = i - k1 * n2, k2 = r / np1, k3 = r - k2 * np1;
            double acc = 0.0;
            for (int j = 0; j < np1; ++j) acc += T[n2 + k2 * np1 + j] * Bm[k1 * n2 + j * np1 + k3];
            A[i] = acc;
        }
        __syncthreads();
        // out[k1,k2,k3] += sum_k3' T3[k3][k3'] C[k1,k2,k3']
        for (int i = tid; i < P; i += blockDim.x) {
            const int k3 = i % np1, base = i - k3;
            double acc = 0.0;
            for (int j = 0; j < np1; ++j) acc += T[2 * n2 + k3 * np1 + j] * A[base + j];
            out[i] += acc;
        }
    }
    __syncthreads();
    double* q = a.qhat64 + static_cast<int64_t>(a.qslot[v]) * P;
    for (int i = tid; i < P; i += blockDim.x) {
        q[i] = out[i];
        if (a.qhat32) a.qhat32[static_cast<int64_t>(a.qslot[v]) * P + i] = static_cast<float>(out[i]);
    }
}

size_t m2m_smem_bytes(int np1) {
    const size_t P = static_cast<size_t>(np1) * np1 * np1;
    return sizeof(double) * (3 * P + 3 * static_cast<size_t>(np1) * np1 + 3 * np1);
}

template <typename F>
size_t upward_smem(int np1) {
    const int pairs = np1 * np1, P = pairs * np1;
    const int G = std::max(1, kThreads / pairs);
    size_t a = sizeof(F) * 3 * np1 * (kTile + 1);
    size_t b = sizeof(F) * static_cast<size_t>(G) * P;
    return std::max(a, b);
}

// Function attributes are per process, not per stream: threads preparing solves of
// different degrees at once must not lower each other's shared-memory limit.  Every call
// therefore sets the same value, the largest any degree needs.
template <typename F>
int upward_smem_max() {
    size_t m = 0;
    for (int np1 = 2; np1 <= BLTC_MAX_DEGREE + 1; ++np1) m = std::max(m, upward_smem<F>(np1));
    return static_cast<int>(m);
}

}  // namespace

void compute_modified_charges(Context* ctx, Tree* st, const Lists* lists, int degree,
                              int precision) {
    require(degree >= 1 && degree <= BLTC_MAX_DEGREE, "modified charges: degree out of range");
    require(precision == BLTC_PRECISION_FP64 || precision == BLTC_PRECISION_MIXED,
            "modified charges: bad precision");
    if (!st->has_q) throw Error(BLTC_ERR_STATE, "modified charges: source tree has no charges");
    if (lists && lists->st != st)
        throw Error(BLTC_ERR_STATE, "modified charges: lists were built for another source tree");
    cudaStream_t s = ctx->stream;
    const int np1 = degree + 1;
    const int P = np1 * np1 * np1;
    const int64_t m = st->n_nodes;

    DBuf<int32_t> flag(ctx, m), pos(ctx, m), tot(ctx, 2);
    if (lists) {
        BLTC_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int32_t) * m, s));
        if (lists->n_app > 0) {
            k_mark_from_lists<<<grid_for(lists->n_app, 256), 256, 0, s>>>(lists->app_ids.p,
                                                                           lists->n_app, flag.p); ++ctx->launches;
        }
    } else {
        k_mark_by_size<<<grid_for(m, 256), 256, 0, s>>>(st->count.p, m, P, flag.p); ++ctx->launches;
    }
    BLTC_LAUNCH_CHECK("upward mark");
    for (int L = 1; L < st->n_levels; ++L) {
        k_propagate<<<grid_for(m, 256), 256, 0, s>>>(st->level.p, st->parent.p, m, L, flag.p); ++ctx->launches;
    }
    BLTC_LAUNCH_CHECK("upward propagate");
    exclusive_scan_i32(ctx, flag.p, pos.p, m, tot.p);
    const int32_t n_slots = *reinterpret_cast<const int32_t*>(ctx->read_words(tot.p, 1));

    st->qslot = DBuf<int32_t>(ctx, m);
    st->q_slots = n_slots;
    st->q_degree = degree;
    st->q_precision = precision;
    st->q_lists = lists ? lists->serial : 0;
    st->qhat64 = DBuf<double>(ctx, static_cast<int64_t>(n_slots) * P);
    st->qhat32 = precision == BLTC_PRECISION_MIXED
                     ? DBuf<float>(ctx, static_cast<int64_t>(n_slots) * P)
                     : DBuf<float>();
    DBuf<int32_t> slot_node(ctx, n_slots), slot_items(ctx, n_slots), item0(ctx, n_slots + 1);
    k_slots<<<grid_for(m, 256), 256, 0, s>>>(flag.p, pos.p, st->count.p, st->nch.p, m, st->qslot.p,
                                             slot_node.p, slot_items.p); ++ctx->launches;
    BLTC_LAUNCH_CHECK("upward slots");
    if (n_slots == 0) return;
    exclusive_scan_i32(ctx, slot_items.p, item0.p, n_slots, tot.p + 1);
    k_append_total<<<1, 1, 0, s>>>(item0.p, n_slots, tot.p + 1); ++ctx->launches;
    const int32_t n_items = reinterpret_cast<const int32_t*>(ctx->read_words(tot.p, 1))[1];
    DBuf<int4> items(ctx, std::max<int32_t>(n_items, 1));
    k_items<<<grid_for(n_slots, 128), 128, 0, s>>>(slot_node.p, item0.p, st->begin.p,
                                                   st->count.p, n_slots, items.p); ++ctx->launches;
    DBuf<double> partial(ctx, static_cast<int64_t>(n_items) * P);

    UpArgs a{};
    a.px = st->px.p;
    a.py = st->py.p;
    a.pz = st->pz.p;
    a.pq = st->pq.p;
    a.begin = st->begin.p;
    a.count = st->count.p;
    a.lo = st->lo.p;
    a.hi = st->hi.p;
    a.cheb_t = ctx->cheb_table(degree);
    a.slot_node = slot_node.p;
    a.items = items.p;
    a.partial = partial.p;
    a.np1 = np1;
    if (n_items > 0) {
        if (precision == BLTC_PRECISION_MIXED) {
            const size_t sm = upward_smem<float>(np1);
            BLTC_CUDA(cudaFuncSetAttribute(k_upward_partial<float>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           upward_smem_max<float>()));
            k_upward_partial<float><<<n_items, kThreads, sm, s>>>(a); ++ctx->launches;
        } else {
            const size_t sm = upward_smem<double>(np1);
            BLTC_CUDA(cudaFuncSetAttribute(k_upward_partial<double>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           upward_smem_max<double>()));
            k_upward_partial<double><<<n_items, kThreads, sm, s>>>(a); ++ctx->launches;
        }
        BLTC_LAUNCH_CHECK("upward partial");
    }
    k_upward_reduce<<<n_slots, 256, 0, s>>>(partial.p, item0.p, P, st->qhat64.p,
                                             precision == BLTC_PRECISION_MIXED ? st->qhat32.p
                                                                               : nullptr); ++ctx->launches;
    BLTC_LAUNCH_CHECK("upward reduce");
    // M2M: marked internal nodes, deepest level first
    const int nl = st->n_levels;
    if (nl > 1) {
        DBuf<int32_t> hist(ctx, 2 * nl + 1), list(ctx, m);
        BLTC_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(int32_t) * (2 * nl + 1), s));
        k_level_hist<<<grid_for(m, 256), 256, 0, s>>>(flag.p, st->nch.p, st->level.p, m, hist.p); ++ctx->launches;
        std::vector<int32_t> h(static_cast<size_t>(nl));
        BLTC_CUDA(cudaMemcpyAsync(h.data(), hist.p, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost, s));
        BLTC_CUDA(cudaStreamSynchronize(s));
        std::vector<int32_t> off(static_cast<size_t>(nl) + 1, 0);
        for (int L = 0; L < nl; ++L) off[L + 1] = off[L] + h[L];
        if (off[nl] > 0) {
            BLTC_CUDA(cudaMemcpyAsync(hist.p + nl, off.data(), sizeof(int32_t) * nl, cudaMemcpyHostToDevice, s));
            BLTC_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(int32_t) * nl, s));
            k_level_fill<<<grid_for(m, 256), 256, 0, s>>>(flag.p, st->nch.p, st->level.p, m, hist.p + nl,
                                                          hist.p, list.p); ++ctx->launches;
            BLTC_CUDA(cudaStreamSynchronize(s));     // `off` lives on the host stack
            M2MArgs ma{st->nch.p, st->child.p, st->qslot.p, st->lo.p, st->hi.p, a.cheb_t, st->qhat64.p,
                       precision == BLTC_PRECISION_MIXED ? st->qhat32.p : nullptr, np1};
            const size_t sm = m2m_smem_bytes(np1);
            BLTC_CUDA(cudaFuncSetAttribute(k_m2m, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           static_cast<int>(m2m_smem_bytes(BLTC_MAX_DEGREE + 1))));
            for (int L = nl - 1; L >= 0; --L) {
                if (h[L] == 0) continue;
                k_m2m<<<h[L], 256, sm, s>>>(ma, list.p + off[L]); ++ctx->launches;
            }
            BLTC_LAUNCH_CHECK("upward m2m");
        }
    }
}

}  // namespace bltc
