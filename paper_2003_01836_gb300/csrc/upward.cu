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
    const int32_t* n_items_dev;       // sized on the device: the item count, else null
    const int32_t* stop;              // sized on the device: the overflow flag
};

// Chebyshev point k of [lo, hi] (Eq. 6 mapped linearly; s_0 = hi and s_n = lo exactly).
__device__ __forceinline__ double cheb_point(const double* t, int k, int n, double lo, double hi) {
    if (k == 0) return hi;
    if (k == n) return lo;
    return __dadd_rn(lo, __dmul_rn(__dmul_rn(0.5, __dadd_rn(t[k], 1.0)), __dsub_rn(hi, lo)));
}

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// P2M (Eq. 12 with Eq. 14-15 factored): the modified charges of one leaf's particle range.
// Phase A turns each particle of a 128-particle tile into its three 1-D factor vectors
// a_l[k] = L_k(y_l) (barycentric form, exact hits of Sec. II-C), with q folded into a_1;
// phase B adds a_1[k1] a_2[k2] a_3[k3] over the tile with one thread per (k1, k2) and
// particle group, n+1 accumulators per thread.
//   Mixed: y - s_k comes from FP32 (hi, lo) pairs of y - c and s_k - c (c the box midpoint),
//   so each particle costs two FP64 operations per dimension instead of n+1; the result has
//   the relative error of rounding the FP64 difference to FP32.  1/(y - s_k) is the SFU
//   reciprocal (w_k is +-1 or +-1/2, so w_k / (y - s_k) is that reciprocal scaled exactly).
//   The barycentric denominator is summed by TwoSum (its terms alternate in sign).
//   FP64: differences, divisions and sums in double.
// Shared memory: fac2 [kTile][np4] (dimension 3, one row per particle padded to a multiple
// of 4 for vector loads), then fac0, fac1 [np1][kTile + 1]; at the end the group-reduction
// buffer [G][P].  NMAX bounds n + 1 (register arrays).
template <typename F, int NMAX>
__global__ void __launch_bounds__(kThreads) k_upward_partial(UpArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int np1 = a.np1, n = np1 - 1;
    const int np4 = (np1 + 3) & ~3;
    const int pairs = np1 * np1;
    const int P = pairs * np1;
    const int G = max(1, kThreads / pairs);
    const int stride = kTile + 1;
    F* fac2 = reinterpret_cast<F*>(smem_raw);
    F* fac0 = fac2 + kTile * np4;
    F* fac1 = fac0 + np1 * stride;
    if (a.n_items_dev && (static_cast<int>(blockIdx.x) >= *a.n_items_dev || *a.stop)) return;
    const int4 it = a.items[blockIdx.x];
    const int node = a.slot_node[it.x];
    const int tid = threadIdx.x;
    const bool active = tid < pairs * G;
    const int p = tid % pairs, g = tid / pairs;
    const int k1 = p / np1, k2 = p % np1;
    F acc[NMAX], lo_acc[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; ++k) acc[k] = lo_acc[k] = F(0);
    __shared__ double s_c[3];
    __shared__ double s_pts[3 * NMAX];          // the cluster's Chebyshev points (FP64 path)
    __shared__ float s_hi[3 * NMAX], s_lo[3 * NMAX];   // s_k - c as FP32 pairs (mixed path)
    if (tid < 3) s_c[tid] = __dmul_rn(0.5, __dadd_rn(a.lo[3 * node + tid], a.hi[3 * node + tid]));
    __syncthreads();
    if (tid < 3 * np1) {
        const int d = tid / np1, k = tid - d * np1;
        const double sk = cheb_point(a.cheb_t, k, n, a.lo[3 * node + d], a.hi[3 * node + d]);
        s_pts[tid] = sk;
        const double r = __dsub_rn(sk, s_c[d]);
        const float h = __double2float_rn(r);
        s_hi[tid] = h;
        s_lo[tid] = __double2float_rn(__dsub_rn(r, static_cast<double>(h)));
    }

    for (int j0 = it.y; j0 < it.z; j0 += kTile) {
        const int m = min(kTile, it.z - j0);
        __syncthreads();
        if (tid < 3 * kTile) {
            const int j = tid % kTile, d = tid / kTile;
            if (j < m) {
                const int pos = j0 + j;
                const double yv = d == 0 ? a.px[pos] : (d == 1 ? a.py[pos] : a.pz[pos]);
                const double qv = d == 0 ? a.pq[pos] : 1.0;
                F vals[NMAX];
#pragma unroll
                for (int k = 0; k < NMAX; ++k) vals[k] = F(0);
                int hit = -1;
                if constexpr (sizeof(F) == 4) {
                    const double r = __dsub_rn(yv, s_c[d]);
                    const float yh = __double2float_rn(r);
                    const float yl = __double2float_rn(__dsub_rn(r, static_cast<double>(yh)));
                    float dk[NMAX];
#pragma unroll
                    for (int k = 0; k < NMAX; ++k) {
                        if (k < np1) {
                            dk[k] = __fadd_rn(__fsub_rn(yh, s_hi[d * np1 + k]), __fsub_rn(yl, s_lo[d * np1 + k]));
                            // |y - s_k| below FLT_MIN is an exact hit (a superset of the FP64
                            // rule |y - s_k| < DBL_MIN, changing L by < 1e-29)
                            if (fabsf(dk[k]) < 1.17549435e-38f && hit < 0) hit = k;
                        }
                    }
                    if (hit < 0) {
                        float den = 0.f, den_lo = 0.f;
#pragma unroll
                        for (int k = 0; k < NMAX; ++k) {
                            if (k < np1) {
                                const float w = ((k == 0 || k == n) ? 0.5f : 1.f) * ((k & 1) ? -1.f : 1.f);
                                vals[k] = w * rcp_approx(dk[k]);
                                const float sum = den + vals[k];
                                const float bb = sum - den;
                                den_lo += (den - (sum - bb)) + (vals[k] - bb);
                                den = sum;
                            }
                        }
                        const float scale = static_cast<float>(qv) / (den + den_lo);
#pragma unroll
                        for (int k = 0; k < NMAX; ++k) vals[k] *= scale;
                    }
                } else {
                    const double* pts = s_pts + d * np1;
                    double dk[NMAX];
#pragma unroll
                    for (int k = 0; k < NMAX; ++k) {
                        if (k < np1) {
                            dk[k] = yv - pts[k];
                            if (fabs(dk[k]) < 2.2250738585072014e-308 && hit < 0) hit = k;
                        }
                    }
                    if (hit < 0) {
                        double den = 0.0;
#pragma unroll
                        for (int k = 0; k < NMAX; ++k) {
                            if (k < np1) {
                                const double w = ((k == 0 || k == n) ? 0.5 : 1.0) * ((k & 1) ? -1.0 : 1.0);
                                vals[k] = w / dk[k];
                                den += vals[k];
                            }
                        }
                        const double scale = qv / den;
#pragma unroll
                        for (int k = 0; k < NMAX; ++k) vals[k] *= scale;
                    }
                }
                if (hit >= 0) {
#pragma unroll
                    for (int k = 0; k < NMAX; ++k) vals[k] = k == hit ? F(qv) : F(0);
                }
                if (d == 2) {
                    F* row = fac2 + j * np4;
#pragma unroll
                    for (int k = 0; k < NMAX; ++k)
                        if (k < np1) row[k] = vals[k];
                    for (int k = np1; k < np4; ++k) row[k] = F(0);
                } else {
                    F* col = (d == 0 ? fac0 : fac1) + j;
#pragma unroll
                    for (int k = 0; k < NMAX; ++k)
                        if (k < np1) col[k * stride] = vals[k];
                }
            }
        }
        __syncthreads();
        if (active) {
            const F* f0 = fac0 + k1 * stride;
            const F* f1 = fac1 + k2 * stride;
            F blk[NMAX + 3];
#pragma unroll
            for (int k = 0; k < NMAX + 3; ++k) blk[k] = F(0);
            for (int j = g; j < m; j += G) {
                const F a12 = f0[j] * f1[j];
                const F* row = fac2 + j * np4;
                if constexpr (sizeof(F) == 4) {
#pragma unroll
                    for (int k4 = 0; k4 < NMAX; k4 += 4) {
                        if (k4 < np1) {
                            const float4 v = *reinterpret_cast<const float4*>(row + k4);
                            blk[k4] += a12 * v.x;
                            blk[k4 + 1] += a12 * v.y;
                            blk[k4 + 2] += a12 * v.z;
                            blk[k4 + 3] += a12 * v.w;
                        }
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < NMAX; ++k)
                        if (k < np1) blk[k] += a12 * row[k];
                }
            }
            if constexpr (sizeof(F) == 4) {
                // fold the tile's FP32 sums into a TwoSum accumulator
#pragma unroll
                for (int k = 0; k < NMAX; ++k) {
                    if (k < np1) {
                        const F sum = acc[k] + blk[k];
                        const F bb = sum - acc[k];
                        lo_acc[k] += (acc[k] - (sum - bb)) + (blk[k] - bb);
                        acc[k] = sum;
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < NMAX; ++k)
                    if (k < np1) acc[k] += blk[k];
            }
        }
    }
    // Sum the particle groups in a fixed order.
    __syncthreads();
    F* red = fac2;                                  // [G][P]
    if (active) {
#pragma unroll
        for (int k = 0; k < NMAX; ++k)
            if (k < np1) red[g * P + p * np1 + k] = acc[k] + lo_acc[k];
    }
    __syncthreads();
    double* out = a.partial + static_cast<int64_t>(blockIdx.x) * P;
    for (int o = tid; o < P; o += kThreads) {
        double sum = 0.0;
        for (int gg = 0; gg < G; ++gg) sum += static_cast<double>(red[gg * P + o]);
        out[o] = sum;
    }
}

__global__ void k_upward_reduce(const double* __restrict__ partial,
                                const int32_t* __restrict__ item0, int P, double* qhat64,
                                float* qhat32, const int32_t* n_slots_dev, const int32_t* stop,
                                int32_t item_cap) {
    const int slot = blockIdx.x;
    if (n_slots_dev && (slot >= *n_slots_dev || *stop)) return;
    const int i0 = item0[slot], i1 = min(item0[slot + 1], item_cap);
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        double s = 0.0;
        for (int i = i0; i < i1; ++i) s += partial[static_cast<int64_t>(i) * P + k];
        qhat64[static_cast<int64_t>(slot) * P + k] = s;
        if (qhat32) qhat32[static_cast<int64_t>(slot) * P + k] = static_cast<float>(s);
    }
}

__global__ void k_mark_from_lists(const int32_t* __restrict__ app_ids, int64_t n,
                                  int32_t* flag, const int32_t* n_dev) {
    if (n_dev && *n_dev < n) n = *n_dev;
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
                        int64_t m, int32_t* qslot, int32_t* slot_node, int32_t* slot_items,
                        int32_t slot_cap, int32_t* cap_flag) {
    int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (v >= m) return;
    if (flag[v] && pos[v] >= slot_cap) {
        // sized on the device and past the capacity: a valid slot keeps every index in range
        atomicOr(cap_flag, 1);
        qslot[v] = slot_cap - 1;
    } else if (flag[v]) {
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
                        const int32_t* __restrict__ count, int64_t n_slots, int4* items,
                        const int32_t* n_slots_dev, int32_t item_cap, int32_t* cap_flag) {
    if (n_slots_dev && *n_slots_dev < n_slots) n_slots = *n_slots_dev;
    int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (s >= n_slots) return;
    const int v = slot_node[s];
    const int b = begin[v], c = count[v];
    // a slot owns items item0[s] .. item0[s+1]-1: none for internal nodes (built by M2M)
    const int i1 = item0[s + 1];
    if (i1 > item_cap) {
        atomicOr(cap_flag, 1);
        return;
    }
    for (int i = item0[s], p0 = b; i < i1; ++i, p0 += kItem)
        items[i] = make_int4(static_cast<int>(s), p0, min(b + c, p0 + kItem), 0);
}

// Sized on the device: the offsets of the levels' marked internal nodes (lev[nl + L]) from
// their counts (lev[L]), zero cursors (lev[2 nl + L]), and the flag when a level holds more
// than the capacity.
__global__ void k_level_offsets(int32_t* lev, int nl, int32_t cap, int32_t* cap_flag) {
    int32_t o = 0;
    for (int L = 0; L < nl; ++L) {
        lev[nl + L] = o;
        lev[2 * nl + L] = 0;
        o += lev[L];
        if (lev[L] > cap) atomicOr(cap_flag, 1);
    }
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
    // sized on the device: per level the count (lev[L]) and the offset in the list
    // (lev[nl + L]) of the marked internal nodes, the capacity per level, and the overflow flag
    const int32_t* lev;
    int nl;
    int32_t cap;
    const int32_t* stop;
};

// The parent of block group j of a launch: nodes[j] (host-driven) or, sized on the device,
// entry p0 + j of level L's part of the list; -1 when beyond the level's count.
__device__ __forceinline__ int m2m_parent(const M2MArgs& a, const int32_t* nodes, int L, int p0, int j) {
    if (!a.lev) return nodes[j];
    if (*a.stop) return -1;
    const int k = p0 + j;
    if (k >= min(a.lev[L], a.cap)) return -1;
    return nodes[a.lev[a.nl + L] + k];
}

// Exact transfer of the children's modified charges to their parent (the parent's Lagrange
// polynomials L^P_k have degree n in each variable, so a child's tensor interpolant (Eq. 4-8)
// reproduces them exactly and, from Eq. 12,
//   qhat^P_k = sum_children sum_k' L^P_k1(s^c_k'1) L^P_k2(s^c_k'2) L^P_k3(s^c_k'3) qhat^c_k').
// GB300's FP64 rate is low per SM, so the work is spread over one block per (parent, child)
// pair: the three (n+1)x(n+1) matrices T_l[k][k'] = L^P_k(s^c_k'l) (barycentric form, exact
// hits as in Sec. II-C), then three mode products into the pair's scratch row.  A second
// kernel adds a parent's rows in child order.  FP64 throughout.
__global__ void __launch_bounds__(256) k_m2m_child(M2MArgs a, const int32_t* __restrict__ nodes,
                                                   double* __restrict__ scratch, int L, int p0) {
    extern __shared__ __align__(16) double m2m_smem[];
    const int v = m2m_parent(a, nodes, L, p0, static_cast<int>(blockIdx.x >> 3)),
              ci = static_cast<int>(blockIdx.x & 7);
    if (v < 0 || ci >= a.nch[v]) return;
    const int c = a.child[8 * v + ci];
    const int np1 = a.np1, n = np1 - 1, P = np1 * np1 * np1, n2 = np1 * np1;
    double* A = m2m_smem;            // child charges, then the second mode product
    double* Bm = A + P;              // first mode product
    double* T = Bm + P;              // [3][np1][np1]
    double* sp = T + 3 * n2;         // parent points [3][np1]
    const int tid = threadIdx.x;
    if (tid < 3 * np1) {
        const int d = tid / np1, k = tid - d * np1;
        sp[tid] = cheb_point(a.cheb_t, k, n, a.lo[3 * v + d], a.hi[3 * v + d]);
    }
    const double* qc = a.qhat64 + static_cast<int64_t>(a.qslot[c]) * P;
    for (int i = tid; i < P; i += blockDim.x) A[i] = qc[i];
    __syncthreads();
    if (tid < 3 * np1) {
        // column k' of T_d: the parent's 1-D Lagrange values at the child's point s^c_k'
        const int d = tid / np1, kp = tid - d * np1;
        const double y = cheb_point(a.cheb_t, kp, n, a.lo[3 * c + d], a.hi[3 * c + d]);
        const double* sv = sp + d * np1;
        double* col = T + d * n2 + kp;            // T_d[k][kp] at col[k * np1]
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
    // row[k1,k2,k3] = sum_k3' T3[k3][k3'] C[k1,k2,k3']
    double* row = scratch + static_cast<int64_t>(blockIdx.x) * P;
    for (int i = tid; i < P; i += blockDim.x) {
        const int k3 = i % np1, base = i - k3;
        double acc = 0.0;
        for (int j = 0; j < np1; ++j) acc += T[2 * n2 + k3 * np1 + j] * A[base + j];
        row[i] = acc;
    }
}

// qhat of each parent: its children's rows added in child order.
__global__ void k_m2m_sum(M2MArgs a, const int32_t* __restrict__ nodes,
                          const double* __restrict__ scratch, int L, int p0) {
    const int v = m2m_parent(a, nodes, L, p0, static_cast<int>(blockIdx.x));
    if (v < 0) return;
    const int nc = a.nch[v];
    const int P = a.np1 * a.np1 * a.np1;
    const double* rows = scratch + static_cast<int64_t>(blockIdx.x) * 8 * P;
    double* q = a.qhat64 + static_cast<int64_t>(a.qslot[v]) * P;
    float* q32 = a.qhat32 ? a.qhat32 + static_cast<int64_t>(a.qslot[v]) * P : nullptr;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        double s = 0.0;
        for (int ci = 0; ci < nc; ++ci) s += rows[static_cast<int64_t>(ci) * P + i];
        q[i] = s;
        if (q32) q32[i] = static_cast<float>(s);
    }
}

size_t m2m_smem_bytes(int np1) {
    const size_t P = static_cast<size_t>(np1) * np1 * np1;
    return sizeof(double) * (2 * P + 3 * static_cast<size_t>(np1) * np1 + 3 * np1);
}

template <typename F>
size_t upward_smem(int np1) {
    const int pairs = np1 * np1, P = pairs * np1, np4 = (np1 + 3) & ~3;
    const int G = std::max(1, kThreads / pairs);
    size_t a = sizeof(F) * (static_cast<size_t>(kTile) * np4 + 2 * static_cast<size_t>(np1) * (kTile + 1));
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

template <typename F, int NMAX>
void launch_partial(const UpArgs& a, int32_t n_items, size_t smem, cudaStream_t s) {
    BLTC_CUDA(cudaFuncSetAttribute(k_upward_partial<F, NMAX>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, upward_smem_max<F>()));
    k_upward_partial<F, NMAX><<<n_items, kThreads, smem, s>>>(a);
}

}  // namespace

void prepare_upward(Context* ctx, Tree* st, const Lists* lists, int degree, int precision,
                    UpwardPlan* up) {
    require(degree >= 1 && degree <= BLTC_MAX_DEGREE, "modified charges: degree out of range");
    require(precision == BLTC_PRECISION_FP64 || precision == BLTC_PRECISION_MIXED,
            "modified charges: bad precision");
    if (!st->has_q) throw Error(BLTC_ERR_STATE, "modified charges: source tree has no charges");
    if (lists && lists->st != st)
        throw Error(BLTC_ERR_STATE, "modified charges: lists were built for another source tree");
    const Caps* caps = st->caps;
    require(!caps || (lists && lists->caps == caps), "modified charges: lists sized differently");
    cudaStream_t s = ctx->stream;
    const int np1 = degree + 1;
    const int P = np1 * np1 * np1;
    const int64_t m = st->n_nodes;
    up->degree = degree;
    up->precision = precision;
    up->caps = caps;

    DBuf<int32_t> flag(ctx, m), pos(ctx, m);
    up->dcount = DBuf<int32_t>(ctx, 2);           // {slots, items}
    int32_t* tot = up->dcount.p;
    int32_t* cap_flag = caps ? caps->flag : nullptr;
    if (lists) {
        BLTC_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int32_t) * m, s));
        if (lists->n_app > 0) {
            k_mark_from_lists<<<grid_for(lists->n_app, 256), 256, 0, s>>>(
                lists->app_ids.p, lists->n_app, flag.p, caps ? lists->dcount.p : nullptr); ++ctx->launches;
        }
    } else {
        k_mark_by_size<<<grid_for(m, 256), 256, 0, s>>>(st->count.p, m, P, flag.p); ++ctx->launches;
    }
    BLTC_LAUNCH_CHECK("upward mark");
    for (int L = 1; L < st->n_levels; ++L) {
        k_propagate<<<grid_for(m, 256), 256, 0, s>>>(st->level.p, st->parent.p, m, L, flag.p); ++ctx->launches;
    }
    BLTC_LAUNCH_CHECK("upward propagate");
    exclusive_scan_i32(ctx, flag.p, pos.p, m, tot);
    const int32_t n_slots = caps ? std::max<int32_t>(1, caps->slots)
                                 : *reinterpret_cast<const int32_t*>(ctx->read_words(tot, 1));

    st->qslot = DBuf<int32_t>(ctx, m);
    st->q_slots = n_slots;
    st->q_degree = degree;
    st->q_precision = precision;
    st->q_lists = lists ? lists->serial : 0;
    st->qhat64 = DBuf<double>(ctx, static_cast<int64_t>(n_slots) * P);
    st->qhat32 = precision == BLTC_PRECISION_MIXED
                     ? DBuf<float>(ctx, static_cast<int64_t>(n_slots) * P)
                     : DBuf<float>();
    up->n_slots = n_slots;
    up->slot_node = DBuf<int32_t>(ctx, n_slots);
    up->item0 = DBuf<int32_t>(ctx, n_slots + 1);
    DBuf<int32_t> slot_items(ctx, n_slots);
    if (caps) BLTC_CUDA(cudaMemsetAsync(slot_items.p, 0, sizeof(int32_t) * n_slots, s));
    k_slots<<<grid_for(m, 256), 256, 0, s>>>(flag.p, pos.p, st->count.p, st->nch.p, m, st->qslot.p,
                                             up->slot_node.p, slot_items.p, n_slots, cap_flag); ++ctx->launches;
    BLTC_LAUNCH_CHECK("upward slots");
    if (!caps && n_slots == 0) return;
    exclusive_scan_i32(ctx, slot_items.p, up->item0.p, n_slots, tot + 1);
    k_append_total<<<1, 1, 0, s>>>(up->item0.p, n_slots, tot + 1); ++ctx->launches;
    const int32_t n_items = caps ? std::max<int32_t>(1, caps->up_items)
                                 : reinterpret_cast<const int32_t*>(ctx->read_words(tot, 1))[1];
    up->n_items = n_items;
    up->items = DBuf<int4>(ctx, std::max<int32_t>(n_items, 1));
    k_items<<<grid_for(n_slots, 128), 128, 0, s>>>(up->slot_node.p, up->item0.p, st->begin.p,
                                                   st->count.p, n_slots, up->items.p,
                                                   caps ? tot : nullptr, caps ? n_items : INT32_MAX,
                                                   cap_flag); ++ctx->launches;
    up->partial = DBuf<double>(ctx, static_cast<int64_t>(n_items) * P);
    ctx->cheb_table(degree);
    // M2M: marked internal nodes per level, deepest level first
    const int nl = st->n_levels;
    up->h.assign(static_cast<size_t>(nl), 0);
    up->off.assign(static_cast<size_t>(nl) + 1, 0);
    if (nl > 1 && caps) {
        // counts, offsets and cursors stay in device memory; the launches cover the capacity
        up->lev = DBuf<int32_t>(ctx, 3 * nl);
        up->list = DBuf<int32_t>(ctx, m);
        BLTC_CUDA(cudaMemsetAsync(up->lev.p, 0, sizeof(int32_t) * 3 * nl, s));
        k_level_hist<<<grid_for(m, 256), 256, 0, s>>>(flag.p, st->nch.p, st->level.p, m, up->lev.p); ++ctx->launches;
        k_level_offsets<<<1, 1, 0, s>>>(up->lev.p, nl, std::max<int32_t>(1, caps->m2m), caps->flag); ++ctx->launches;
        k_level_fill<<<grid_for(m, 256), 256, 0, s>>>(flag.p, st->nch.p, st->level.p, m, up->lev.p + nl,
                                                      up->lev.p + 2 * nl, up->list.p); ++ctx->launches;
        BLTC_LAUNCH_CHECK("upward levels");
        const int32_t hmax = std::max<int32_t>(1, caps->m2m);
        for (int L = 0; L < nl; ++L) up->h[L] = hmax;
        up->chunk = static_cast<int32_t>(std::max<int64_t>(
            1, std::min<int64_t>(hmax, (int64_t(32) << 20) / (8 * static_cast<int64_t>(P) * 8))));
        up->scratch = DBuf<double>(ctx, static_cast<int64_t>(up->chunk) * 8 * P);
        up->off[nl] = 1;
    } else if (nl > 1) {
        DBuf<int32_t> hist(ctx, 2 * nl + 1);
        up->list = DBuf<int32_t>(ctx, m);
        BLTC_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(int32_t) * (2 * nl + 1), s));
        k_level_hist<<<grid_for(m, 256), 256, 0, s>>>(flag.p, st->nch.p, st->level.p, m, hist.p); ++ctx->launches;
        BLTC_CUDA(cudaMemcpyAsync(up->h.data(), hist.p, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost, s));
        BLTC_CUDA(cudaStreamSynchronize(s));
        for (int L = 0; L < nl; ++L) up->off[L + 1] = up->off[L] + up->h[L];
        if (up->off[nl] > 0) {
            BLTC_CUDA(cudaMemcpyAsync(hist.p + nl, up->off.data(), sizeof(int32_t) * nl, cudaMemcpyHostToDevice, s));
            BLTC_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(int32_t) * nl, s));
            k_level_fill<<<grid_for(m, 256), 256, 0, s>>>(flag.p, st->nch.p, st->level.p, m, hist.p + nl,
                                                          hist.p, up->list.p); ++ctx->launches;
            BLTC_CUDA(cudaStreamSynchronize(s));     // the offsets are read from host memory
            // scratch rows for 8 children per parent, at most ~32 MB at a time
            int32_t hmax = 0;
            for (int L = 0; L < nl; ++L) hmax = std::max(hmax, up->h[L]);
            up->chunk = static_cast<int32_t>(std::max<int64_t>(
                1, std::min<int64_t>(hmax, (int64_t(32) << 20) / (8 * static_cast<int64_t>(P) * 8))));
            up->scratch = DBuf<double>(ctx, static_cast<int64_t>(up->chunk) * 8 * P);
        }
    }
}

void run_upward(Context* ctx, Tree* st, const UpwardPlan& up) {
    if (up.n_slots == 0) return;
    cudaStream_t s = ctx->stream;
    const int degree = up.degree, precision = up.precision;
    const int np1 = degree + 1;
    const int P = np1 * np1 * np1;
    const Caps* caps = up.caps;
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
    a.slot_node = up.slot_node.p;
    a.items = up.items.p;
    a.partial = up.partial.p;
    a.np1 = np1;
    a.n_items_dev = caps ? up.dcount.p + 1 : nullptr;
    a.stop = caps ? caps->flag : nullptr;
    if (up.n_items > 0) {
        if (precision == BLTC_PRECISION_MIXED) {
            const size_t sm = upward_smem<float>(np1);
            if (np1 <= 9) launch_partial<float, 9>(a, up.n_items, sm, s);
            else launch_partial<float, BLTC_MAX_DEGREE + 1>(a, up.n_items, sm, s);
        } else {
            const size_t sm = upward_smem<double>(np1);
            if (np1 <= 9) launch_partial<double, 9>(a, up.n_items, sm, s);
            else launch_partial<double, BLTC_MAX_DEGREE + 1>(a, up.n_items, sm, s);
        }
        ++ctx->launches;
        BLTC_LAUNCH_CHECK("upward partial");
    }
    k_upward_reduce<<<up.n_slots, 256, 0, s>>>(up.partial.p, up.item0.p, P, st->qhat64.p,
                                                precision == BLTC_PRECISION_MIXED ? st->qhat32.p : nullptr,
                                                caps ? up.dcount.p : nullptr, a.stop,
                                                caps ? up.n_items : INT32_MAX); ++ctx->launches;
    BLTC_LAUNCH_CHECK("upward reduce");
    const int nl = static_cast<int>(up.h.size());
    if (nl > 1 && up.off[nl] > 0) {
        M2MArgs ma{st->nch.p, st->child.p, st->qslot.p, st->lo.p, st->hi.p, a.cheb_t, st->qhat64.p,
                   precision == BLTC_PRECISION_MIXED ? st->qhat32.p : nullptr, np1,
                   caps ? up.lev.p : nullptr, nl, caps ? std::max<int32_t>(1, caps->m2m) : 0, a.stop};
        const size_t sm = m2m_smem_bytes(np1);
        BLTC_CUDA(cudaFuncSetAttribute(k_m2m_child, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(m2m_smem_bytes(BLTC_MAX_DEGREE + 1))));
        for (int L = nl - 1; L >= 0; --L) {
            for (int32_t p0 = 0; p0 < up.h[L]; p0 += up.chunk) {
                const int32_t np = std::min(up.chunk, up.h[L] - p0);
                // host-driven: the chunk's parents; sized on the device: the list, read by level
                const int32_t* nodes = caps ? up.list.p : up.list.p + up.off[L] + p0;
                k_m2m_child<<<8 * np, 256, sm, s>>>(ma, nodes, up.scratch.p, L, p0); ++ctx->launches;
                k_m2m_sum<<<np, 256, 0, s>>>(ma, nodes, up.scratch.p, L, p0); ++ctx->launches;
            }
        }
        BLTC_LAUNCH_CHECK("upward m2m");
    }
}

void compute_modified_charges(Context* ctx, Tree* st, const Lists* lists, int degree,
                              int precision) {
    UpwardPlan up;
    prepare_upward(ctx, st, lists, degree, precision, &up);
    run_upward(ctx, st, up);
}

}  // namespace bltc
