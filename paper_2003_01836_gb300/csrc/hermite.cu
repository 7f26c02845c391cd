// hermite.cu -- the barycentric Hermite treecode (future work of Sec. V), FP64 or mixed precision.
//
// Reading (the paper names the method without defining it): on the n+1 Chebyshev points of
// Eq. 6 a cluster's kernel is interpolated with values and first derivatives, the classical
// Hermite basis H_k(y) = (1 - 2 L_k'(s_k)(y - s_k)) L_k(y)^2, K_k(y) = (y - s_k) L_k(y)^2
// with L_k of Eq. 4 (exact hits of Sec. II-C give H = e_m, K = 0), which reproduces degree
// 2n+1.  In three variables the 8 mixed derivatives a in {0,1}^3 enter:
//     phi(x_i) ~ sum_k sum_a D^a G(x_i, s_k) qhat^a_k,
//     qhat^a_k = sum_{y_j in C} q_j B^{a1}_{k1}(y_j1) B^{a2}_{k2}(y_j2) B^{a3}_{k3}(y_j3),
// B^0 = H, B^1 = K.  The MAC is Eq. 13 with the size test 8 (n+1)^3 < N_C, which the list
// builder applies when given degree 2n+1 ((2n+2)^3 = 8 (n+1)^3).
//
// GPU mapping: the lists and the work plan are the treecode's; the modified charges of each
// approximated cluster are summed from its particles in FP64 (k_herm_partial, one block per
// chunk of a cluster's particles, a fixed-order reduction per cluster, an FP32 copy for the
// mixed path); the sweep's far field evaluates the 8 derivative terms per point
// (far_hermite_fp64, or far_hermite_mixed in FP32 on batch-relative coordinates beside the
// treecode's mixed near field).
#include <algorithm>

#include "internal.cuh"

namespace bltc {
namespace {

constexpr int kHThreads = 512;
constexpr int kHTile = 64;                 // particles per factor tile
constexpr int kHItem = 2048;               // particles per item
constexpr int kHMax = 8;                   // n + 1 <= 8

__device__ __forceinline__ double cheb_pt(const double* t, int k, int n, double lo, double hi) {
    if (k == 0) return hi;
    if (k == n) return lo;
    return __dadd_rn(lo, __dmul_rn(__dmul_rn(0.5, __dadd_rn(t[k], 1.0)), __dsub_rn(hi, lo)));
}

__global__ void k_h_mark(const int32_t* __restrict__ app_ids, int64_t n, int32_t* flag) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) flag[app_ids[i]] = 1;
}

__global__ void k_h_slots(const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                          const int32_t* __restrict__ count, int64_t m, int32_t* qslot, int32_t* slot_node,
                          int32_t* slot_items) {
    const int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= m) return;
    if (flag[v]) {
        qslot[v] = pos[v];
        slot_node[pos[v]] = static_cast<int32_t>(v);
        slot_items[pos[v]] = (count[v] + kHItem - 1) / kHItem;
    } else {
        qslot[v] = -1;
    }
}

__global__ void k_h_total(int32_t* off, int64_t n, const int32_t* total) { off[n] = *total; }

__global__ void k_h_items(const int32_t* __restrict__ slot_node, const int32_t* __restrict__ item0,
                          const int32_t* __restrict__ begin, const int32_t* __restrict__ count, int64_t n_slots,
                          int4* items) {
    const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= n_slots) return;
    const int v = slot_node[s];
    const int b = begin[v], c = count[v];
    const int i1 = item0[s + 1];
    for (int i = item0[s], p0 = b; i < i1; ++i, p0 += kHItem)
        items[i] = make_int4(static_cast<int>(s), p0, min(b + c, p0 + kHItem), 0);
}

// One item: the 8 (n+1)^3 sums of a chunk of a cluster's particles.  Phase A tabulates, per
// particle and dimension, H_k and K_k (q folded into the first dimension); phase B gives each
// thread one (a, k1, k2) and a share of the particles, n+1 accumulators over k3.
__global__ void __launch_bounds__(kHThreads) k_herm_partial(const double* __restrict__ px, const double* __restrict__ py,
                                                          const double* __restrict__ pz, const double* __restrict__ pq,
                                                          const double* __restrict__ lo, const double* __restrict__ hi,
                                                          const double* __restrict__ cheb_t,
                                                          const int32_t* __restrict__ slot_node,
                                                          const int4* __restrict__ items, int np1, double* partial) {
    __shared__ double fh[3][kHMax][kHTile], fk[3][kHMax][kHTile];
    __shared__ double s_pts[3][kHMax], s_dl[3][kHMax];
    extern __shared__ double red[];                      // [G][8 P]
    const int n = np1 - 1, n2 = np1 * np1, P = n2 * np1;
    const int combos = 8 * n2;
    const int G = max(1, kHThreads / combos);
    const int tid = threadIdx.x;
    const bool active = tid < combos * G;
    const int cmb = tid % combos, g = tid / combos;
    const int a = cmb / n2, r = cmb - a * n2, k1 = r / np1, k2 = r - k1 * np1;
    const int4 it = items[blockIdx.x];
    const int node = slot_node[it.x];
    if (tid < 3 * np1) {
        const int d = tid / np1, k = tid - d * np1;
        s_pts[d][k] = cheb_pt(cheb_t, k, n, lo[3 * node + d], hi[3 * node + d]);
    }
    __syncthreads();
    if (tid < 3 * np1) {
        const int d = tid / np1, k = tid - d * np1;
        double dl = 0.0;
        for (int j = 0; j < np1; ++j)
            if (j != k) dl += 1.0 / (s_pts[d][k] - s_pts[d][j]);
        s_dl[d][k] = dl;
    }
    double acc[kHMax];
#pragma unroll
    for (int k = 0; k < kHMax; ++k) acc[k] = 0.0;
    for (int j0 = it.y; j0 < it.z; j0 += kHTile) {
        const int m = min(kHTile, it.z - j0);
        __syncthreads();
        if (tid < 3 * kHTile) {
            const int j = tid % kHTile, d = tid / kHTile;
            if (j < m) {
                const int pos = j0 + j;
                const double y = d == 0 ? px[pos] : (d == 1 ? py[pos] : pz[pos]);
                const double qv = d == 0 ? pq[pos] : 1.0;
                int hit = -1;
                for (int k = 0; k < np1; ++k)
                    if (hit < 0 && fabs(y - s_pts[d][k]) < 2.2250738585072014e-308) hit = k;
                if (hit >= 0) {
                    for (int k = 0; k < np1; ++k) {
                        fh[d][k][j] = k == hit ? qv : 0.0;
                        fk[d][k][j] = 0.0;
                    }
                } else {
                    double l[kHMax], den = 0.0;
                    for (int k = 0; k < np1; ++k) {
                        const double w = ((k == 0 || k == n) ? 0.5 : 1.0) * ((k & 1) ? -1.0 : 1.0);
                        l[k] = w / (y - s_pts[d][k]);
                        den += l[k];
                    }
                    for (int k = 0; k < np1; ++k) {
                        const double lk = l[k] / den;
                        const double l2 = lk * lk, dy = y - s_pts[d][k];
                        fh[d][k][j] = qv * ((1.0 - 2.0 * s_dl[d][k] * dy) * l2);
                        fk[d][k][j] = qv * (dy * l2);
                    }
                }
            }
        }
        __syncthreads();
        if (active) {
            const double* f1 = (a & 4) ? fk[0][k1] : fh[0][k1];
            const double* f2 = (a & 2) ? fk[1][k2] : fh[1][k2];
            for (int j = g; j < m; j += G) {
                const double a12 = f1[j] * f2[j];
#pragma unroll
                for (int k = 0; k < kHMax; ++k)
                    if (k < np1) acc[k] += a12 * ((a & 1) ? fk[2][k][j] : fh[2][k][j]);
            }
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int k = 0; k < kHMax; ++k)
            if (k < np1) red[static_cast<int64_t>(g) * 8 * P + a * P + (k1 * np1 + k2) * np1 + k] = acc[k];
    }
    __syncthreads();
    double* out = partial + static_cast<int64_t>(blockIdx.x) * 8 * P;
    for (int o = tid; o < 8 * P; o += kHThreads) {
        double sum = 0.0;
        for (int gg = 0; gg < G; ++gg) sum += red[static_cast<int64_t>(gg) * 8 * P + o];
        out[o] = sum;
    }
}

__global__ void k_h_reduce(const double* __restrict__ partial, const int32_t* __restrict__ item0, int Q,
                           double* qh, float* qh32) {
    const int slot = blockIdx.x;
    const int i0 = item0[slot], i1 = item0[slot + 1];
    for (int k = threadIdx.x; k < Q; k += blockDim.x) {
        double sum = 0.0;
        for (int i = i0; i < i1; ++i) sum += partial[static_cast<int64_t>(i) * Q + k];
        qh[static_cast<int64_t>(slot) * Q + k] = sum;
        if (qh32) qh32[static_cast<int64_t>(slot) * Q + k] = __double2float_rn(sum);
    }
}

}  // namespace

void solve_device_hermite(Context* c, const double* x, const double* y, const double* z, const double* q,
                          int64_t n, const bltc_params& p, double* phi) {
    require(p.precision == BLTC_PRECISION_FP64 || p.precision == BLTC_PRECISION_MIXED, "hermite: bad precision");
    const bool mixed = p.precision == BLTC_PRECISION_MIXED;
    require(p.degree >= 1 && 2 * p.degree + 1 <= BLTC_MAX_DEGREE, "hermite: degree must be in [1, 7]");
    require(p.kernel == BLTC_KERNEL_COULOMB || p.kernel == BLTC_KERNEL_YUKAWA,
            "hermite: the Coulomb and Yukawa kernels only (derivatives are built in)");
    cudaStream_t s = c->stream;
    const int np1 = p.degree + 1, P = np1 * np1 * np1, Q = 8 * P;
    c->mark(Context::kStart);
    Tree st, btree;
    build_tree(c, x, y, z, q, n, p.leaf_size, &st);
    const Tree* bt = &st;
    if (p.batch_size != p.leaf_size) {
        build_tree(c, x, y, z, nullptr, n, p.batch_size, &btree);
        bt = &btree;
    }
    c->mark(Context::kTrees);
    Lists L;
    build_lists(c, bt, &st, p.theta, 2 * p.degree + 1, &L);       // size test 8 (n+1)^3 < N_C
    c->mark(Context::kLists);
    // Hermite modified charges of every approximated cluster
    const int64_t m = st.n_nodes;
    DBuf<int32_t> flag(c, m), pos(c, m), qslot(c, m), tot(c, 4);
    BLTC_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int32_t) * m, s));
    if (L.n_app > 0) {
        k_h_mark<<<grid_for(L.n_app, 256), 256, 0, s>>>(L.app_ids.p, L.n_app, flag.p); ++c->launches;
    }
    exclusive_scan_i32(c, flag.p, pos.p, m, tot.p);
    const int32_t n_slots = *reinterpret_cast<const int32_t*>(c->read_words(tot.p, 1));
    DBuf<int32_t> slot_node(c, n_slots), slot_items(c, n_slots), item0(c, n_slots + 1);
    k_h_slots<<<grid_for(m, 256), 256, 0, s>>>(flag.p, pos.p, st.count.p, m, qslot.p, slot_node.p,
                                               slot_items.p); ++c->launches;
    DBuf<double> qh(c, static_cast<int64_t>(n_slots) * Q);
    DBuf<float> qh32(c, mixed ? static_cast<int64_t>(n_slots) * Q : 0);
    if (n_slots > 0) {
        exclusive_scan_i32(c, slot_items.p, item0.p, n_slots, tot.p + 1);
        k_h_total<<<1, 1, 0, s>>>(item0.p, n_slots, tot.p + 1); ++c->launches;
        const int32_t n_items = reinterpret_cast<const int32_t*>(c->read_words(tot.p, 1))[1];
        DBuf<int4> items(c, n_items);
        k_h_items<<<grid_for(n_slots, 128), 128, 0, s>>>(slot_node.p, item0.p, st.begin.p, st.count.p, n_slots,
                                                         items.p); ++c->launches;
        DBuf<double> partial(c, static_cast<int64_t>(n_items) * Q);
        const int G = std::max(1, kHThreads / (8 * np1 * np1));
        const size_t smem = sizeof(double) * static_cast<size_t>(G) * Q;
        BLTC_CUDA(cudaFuncSetAttribute(k_herm_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
        k_herm_partial<<<n_items, kHThreads, smem, s>>>(st.px.p, st.py.p, st.pz.p, st.pq.p, st.lo.p, st.hi.p,
                                                        c->cheb_table(p.degree), slot_node.p, items.p, np1,
                                                        partial.p); ++c->launches;
        k_h_reduce<<<n_slots, 256, 0, s>>>(partial.p, item0.p, Q, qh.p, mixed ? qh32.p : nullptr); ++c->launches;
        BLTC_LAUNCH_CHECK("hermite charges");
    }
    c->mark(Context::kUpward);
    evaluate_hermite(c, &L, bt, &st, p, qh.p, mixed ? qh32.p : nullptr, qslot.p, phi);
}

}  // namespace bltc
