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
#include <vector>

#include "internal.cuh"

namespace bltc {
namespace {

constexpr int kThreads = 256;
constexpr int kSrcTile32 = 2048;      // float4 sources per staged tile (32 KB)
constexpr int kSrcTile64 = 1280;      // D4 sources per staged tile (40 KB)
constexpr int kSmemBytes = 40960;     // also holds 3(n+1) + (n+1)^3 doubles for n <= 16
constexpr int kItemsPerBlock = 16;    // work items per resident block (load balance)
constexpr int kBlock = 32;            // terms summed in FP32 before a TwoSum fold

struct SweepArgs {
    // target batches
    const int32_t* b_leaves;
    const int32_t* b_begin;
    const int32_t* b_count;
    const double* b_center;
    const double *tx, *ty, *tz;
    // source clusters
    const int32_t* s_begin;
    const int32_t* s_count;
    const double* s_lo;
    const double* s_hi;
    const double *sx, *sy, *sz, *sq;
    const int32_t* qslot;
    const double* qhat64;
    const float* qhat32;
    const double* cheb_t;
    int np1;
    // lists and items
    const int32_t* app_off;
    const int32_t* app_ids;
    const int32_t* dir_off;
    const int32_t* dir_ids;
    const uint8_t* dir_sel;    // per direct entry: bit 0 = r^2 == 0 possible, bit 1 = close pairs possible
    const float* dir_tau2;     // per direct entry: pairs closer than this (r^2) are redone in FP64
    const int64_t* dir_moff;   // per direct entry: offset of its mutual row in mpart, or -1
    double* mpart;             // mutual rows: potentials a batch's particles induce on a partner's
    const int4* items;
    const int64_t* part_off;
    double* partials;
    int n_items;
    unsigned int* counter;
    // kernel
    int kernel;
    double kappa;
    float neg_kappa_log2e;
};

__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Knuth's TwoSum: hi + lo += v exactly up to the rounding of lo (no magnitude ordering
// needed).  Folds a short FP32 block sum into a compensated FP32 accumulator.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

__device__ __forceinline__ double cheb_point(const double* t, int k, int n, double lo, double hi) {
    if (k == 0) return hi;
    if (k == n) return lo;
    return __dadd_rn(lo, __dmul_rn(__dmul_rn(0.5, __dadd_rn(t[k], 1.0)), __dsub_rn(hi, lo)));
}

// ---- mixed precision ------------------------------------------------------------------

// G(r) without the charge: 1/r, or e^{-kappa r}/r as 2^{-kappa log2(e) r} / r.  The charge
// multiplies last in both kernels, so kappa = 0 reproduces Coulomb bit for bit.
template <int KER>
__device__ __forceinline__ float ri_mixed(float r2, float nkl2e) {
    float ri = rsqrt_approx(r2);
    if (KER == BLTC_KERNEL_YUKAWA) ri *= ex2_approx(nkl2e * (r2 * ri));
    return ri;
}

// Packed FP32x2 arithmetic (FADD2 / FMUL2 / FFMA2 on sm_100 and later): one instruction
// works on two targets, which halves the FMA-pipe issue slots per interaction so that the
// SFU (one MUFU.RSQ per interaction) becomes the binding pipe.  Each lane of a packed
// operation rounds exactly like the scalar operation, so both paths give identical bits.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <int KER>
__device__ __forceinline__ float2 ri2_mixed(float2 r2, float nkl2e, bool skip_zero) {
    float2 ri = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
    if (skip_zero) {
        ri.x = r2.x > 0.f ? ri.x : 0.f;
        ri.y = r2.y > 0.f ? ri.y : 0.f;
    }
    if (KER == BLTC_KERNEL_YUKAWA) {
        const float2 a = mul2(make_float2(nkl2e, nkl2e), mul2(r2, ri));
        ri = mul2(ri, make_float2(ex2_approx(a.x), ex2_approx(a.y)));
    }
    return ri;
}

// Targets of one thread: 8 values per coordinate relative to the batch centre, negated and
// paired: (-x[2v], -x[2v+1]), so s - x is one packed add.
constexpr int kT = 8;                 // targets per thread (even)
constexpr int kH = kT / 2;
constexpr int kMinBlocks = 2;         // resident blocks per SM the register budget must allow
// Dynamic shared memory of the mixed sweep: the staging area, then each thread's kT FP64
// partial potentials ([kT][kThreads], touched once per cluster or tile), which would
// otherwise hold 16 registers through the inner loops.
constexpr int kNearTile = kSrcTile32 / 2;    // sources per staged near-field tile
// then, for mutual pairs, one FP32 slot per warp and staged source: [warp][kNearTile]
constexpr int kAccBytes = kThreads * kT * static_cast<int>(sizeof(double));
constexpr int kMixedSmem = kSmemBytes + kAccBytes + (kThreads / 32) * kNearTile * static_cast<int>(sizeof(float));
constexpr uint8_t kSelZero = 1, kSelClose = 2, kSelMutual = 4, kSelSkip = 8;
struct Targets {
    float2 x[kH], y[kH], z[kH];
};

// Source groups.  A block is 256 threads x kT targets.  A batch of nb targets uses G groups
// of 256/G threads (G = 1, 2, 4, 8 as nb shrinks below 256*kT, 128*kT, 64*kT): every group covers
// all targets of the batch and takes every G-th block of work of each cluster (blocks of
// kBlock sources in the near field, (k1, k2) rows of the proxy grid in the far field).  Each
// group keeps its own partial potentials; they are added in group order at the end of the
// item, so the result is fixed by the batch alone.
__device__ __forceinline__ int groups_for(int nb) {
    return nb > 128 * kT ? 1 : (nb > 64 * kT ? 2 : (nb > 32 * kT ? 4 : 8));
}

// Near field (Eq. 9) of cluster C.  Shared memory holds each staged source as two float4:
// (x, x, y, y) and (z, z, q, q), relative to the batch centre, so a packed operand is one
// aligned register pair.  Sums run over blocks of kBlock sources in FP32, folded into a
// TwoSum accumulator, then into FP64 per staged tile.
template <int KER, bool SEL, bool CHECK>
__device__ void near_mixed(const SweepArgs& a, int C, float tau2, const double cb[3], const Targets& tg,
                           double* acc, float4* sm, int g, int G, int tb, int nb, int t0,
                           int l, int tpg) {
    constexpr int kTile = kNearTile;
    const int cs = a.s_begin[C], nc = a.s_count[C];
    for (int j0 = 0; j0 < nc; j0 += kTile) {
        const int m = min(kTile, nc - j0);
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += kThreads) {
            const int p = cs + j0 + j;
            const float sx = __double2float_rn(a.sx[p] - cb[0]);
            const float sy = __double2float_rn(a.sy[p] - cb[1]);
            const float sz = __double2float_rn(a.sz[p] - cb[2]);
            const float sq = __double2float_rn(a.sq[p]);
            sm[2 * j] = make_float4(sx, sx, sy, sy);
            sm[2 * j + 1] = make_float4(sz, sz, sq, sq);
        }
        __syncthreads();
        float hi[kT], lo[kT];
#pragma unroll
        for (int u = 0; u < kT; ++u) hi[u] = lo[u] = 0.f;
        for (int jb = g * kBlock; jb < m; jb += G * kBlock) {
            const int je = min(jb + kBlock, m);
            float2 f[kH];
#pragma unroll
            for (int v = 0; v < kH; ++v) f[v] = make_float2(0.f, 0.f);
            float rmin = 3.0e38f;      // smallest non-zero r^2 this thread met in the block
#pragma unroll 4
            for (int j = jb; j < je; ++j) {
                const float4 p0 = sm[2 * j], p1 = sm[2 * j + 1];
                const float2 sx = make_float2(p0.x, p0.y), sy = make_float2(p0.z, p0.w);
                const float2 sz = make_float2(p1.x, p1.y), sq = make_float2(p1.z, p1.w);
#pragma unroll
                for (int v = 0; v < kH; ++v) {
                    const float2 dx = add2(sx, tg.x[v]);
                    const float2 dy = add2(sy, tg.y[v]);
                    const float2 dz = add2(sz, tg.z[v]);
                    const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
                    if (CHECK) {
                        if (SEL) {
                            rmin = fminf(rmin, r2.x > 0.f ? r2.x : 3.0e38f);
                            rmin = fminf(rmin, r2.y > 0.f ? r2.y : 3.0e38f);
                        } else {
                            rmin = fminf(rmin, fminf(r2.x, r2.y));
                        }
                    }
                    f[v] = fma2(sq, ri2_mixed<KER>(r2, a.neg_kappa_log2e, SEL), f[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < kH; ++v) {
                two_sum_add(hi[2 * v], lo[2 * v], f[v].x);
                two_sum_add(hi[2 * v + 1], lo[2 * v + 1], f[v].y);
            }
            if (CHECK && rmin < tau2) {
                // Close pairs: their FP32 distance carries the rounding of the batch-relative
                // coordinates (about 2^-23 of the box extent), far too much relative to a tiny
                // r.  Recompute those terms from the FP64 coordinates and add the difference.
                for (int j = jb; j < je; ++j) {
                    const float4 p0 = sm[2 * j], p1 = sm[2 * j + 1];
#pragma unroll
                    for (int u = 0; u < kT; ++u) {
                        const float2 ptx = tg.x[u / 2], pty = tg.y[u / 2], ptz = tg.z[u / 2];
                        const float dx = p0.x + ((u & 1) ? ptx.y : ptx.x);
                        const float dy = p0.z + ((u & 1) ? pty.y : pty.x);
                        const float dz = p1.x + ((u & 1) ? ptz.y : ptz.x);
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        if (r2 > 0.f && r2 < tau2) {
                            const int t = min(t0 + l + tpg * u, nb - 1);
                            const int ps = cs + j0 + j;
                            const double ex = a.sx[ps] - a.tx[tb + t], ey = a.sy[ps] - a.ty[tb + t];
                            const double ez = a.sz[ps] - a.tz[tb + t];
                            const double r2d = ex * ex + ey * ey + ez * ez;
                            double rid = rsqrt(r2d);
                            if (KER == BLTC_KERNEL_YUKAWA) rid *= exp(-a.kappa * (r2d * rid));
                            float ri = rsqrt_approx(r2);
                            if (KER == BLTC_KERNEL_YUKAWA) ri *= ex2_approx(a.neg_kappa_log2e * (r2 * ri));
                            const double corr = a.sq[ps] * rid - static_cast<double>(p1.z * ri);
                            lo[u] += static_cast<float>(corr);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kT; ++u) acc[u * kThreads] += static_cast<double>(hi[u]) + static_cast<double>(lo[u]);
    }
}

// Sum over the 32 lanes of eight values per lane, v[s] for sources s = 0..7, by recursive
// halving: 4 + 2 + 1 exchanges leave lane l with the sum over eight lanes of source l >> 2,
// two more complete it.  Nine shuffles instead of 40; the order of the additions is fixed.
__device__ __forceinline__ float warp_sum8(const float (&v)[8], int lane) {
    const unsigned full = 0xffffffffu;
    const bool h4 = (lane >> 4) & 1, h3 = (lane >> 3) & 1, h2 = (lane >> 2) & 1;
    float w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = h4 ? v[i] : v[i + 4];
        const float keep = h4 ? v[i + 4] : v[i];
        w[i] = keep + __shfl_xor_sync(full, send, 16);
    }
    float x[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = h3 ? w[i] : w[i + 2];
        const float keep = h3 ? w[i + 2] : w[i];
        x[i] = keep + __shfl_xor_sync(full, send, 8);
    }
    float y = (h2 ? x[1] : x[0]) + __shfl_xor_sync(full, h2 ? x[0] : x[1], 4);
    y += __shfl_xor_sync(full, y, 1);
    y += __shfl_xor_sync(full, y, 2);
    return y;
}

// Near field of a mutual pair: batch B (the targets) and leaf C are each in the other's
// direct list and are the same particles as sources and targets, so one evaluation of
// G(x_i, y_j) serves both phi_i += G q_j (as in near_mixed) and phi_j += G q_i (Eq. 9 for C's
// own batch, whose list entry for B is skipped).  The second sum runs over B's targets,
// which sit in different lanes: per source, each lane adds its 8 targets' q_i G in FP32, the
// warp adds its lanes (warp_sum8), and after the tile the group's warps are added in warp
// order into C's mutual row (FP64), so the result does not depend on scheduling.
template <int KER, bool SEL, bool CHECK>
__device__ void near_mutual(const SweepArgs& a, int C, float tau2, const double cb[3], const Targets& tg,
                            double* acc, float4* sm, float* sbuf, double* mrow, int g, int G, int tb,
                            int nb, int t0, int l, int tpg) {
    constexpr int kTile = kNearTile;
    const int cs = a.s_begin[C], nc = a.s_count[C];
    const int lane = static_cast<int>(threadIdx.x) & 31, warp = static_cast<int>(threadIdx.x) >> 5;
    const int wpg = tpg >> 5;                            // warps per group
    // this thread's target charges (0 for the padding slots past the batch)
    float2 qt[kH];
#pragma unroll
    for (int u = 0; u < kT; ++u) {
        const int t = t0 + l + tpg * u;
        const float qv = t < nb ? __double2float_rn(a.sq[tb + t]) : 0.f;
        if (u & 1) qt[u / 2].y = qv; else qt[u / 2].x = qv;
    }
    for (int j0 = 0; j0 < nc; j0 += kTile) {
        const int m = min(kTile, nc - j0);
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += kThreads) {
            const int p = cs + j0 + j;
            const float sx = __double2float_rn(a.sx[p] - cb[0]);
            const float sy = __double2float_rn(a.sy[p] - cb[1]);
            const float sz = __double2float_rn(a.sz[p] - cb[2]);
            const float sq = __double2float_rn(a.sq[p]);
            sm[2 * j] = make_float4(sx, sx, sy, sy);
            sm[2 * j + 1] = make_float4(sz, sz, sq, sq);
        }
        __syncthreads();
        float hi[kT], lo[kT];
#pragma unroll
        for (int u = 0; u < kT; ++u) hi[u] = lo[u] = 0.f;
        for (int jb = g * kBlock; jb < m; jb += G * kBlock) {
            const int je = min(jb + kBlock, m);
            float2 f[kH];
#pragma unroll
            for (int v = 0; v < kH; ++v) f[v] = make_float2(0.f, 0.f);
            float rmin = 3.0e38f;
            for (int j8 = jb; j8 < je; j8 += 8) {
                float gs[8];
#pragma unroll
                for (int s8 = 0; s8 < 8; ++s8) {
                    gs[s8] = 0.f;
                    if (j8 + s8 < je) {
                        const float4 p0 = sm[2 * (j8 + s8)], p1 = sm[2 * (j8 + s8) + 1];
                        const float2 sx = make_float2(p0.x, p0.y), sy = make_float2(p0.z, p0.w);
                        const float2 sz = make_float2(p1.x, p1.y), sq = make_float2(p1.z, p1.w);
                        float2 g2 = make_float2(0.f, 0.f);
#pragma unroll
                        for (int v = 0; v < kH; ++v) {
                            const float2 dx = add2(sx, tg.x[v]);
                            const float2 dy = add2(sy, tg.y[v]);
                            const float2 dz = add2(sz, tg.z[v]);
                            const float2 r2 = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
                            if (CHECK) {
                                if (SEL) {
                                    rmin = fminf(rmin, r2.x > 0.f ? r2.x : 3.0e38f);
                                    rmin = fminf(rmin, r2.y > 0.f ? r2.y : 3.0e38f);
                                } else {
                                    rmin = fminf(rmin, fminf(r2.x, r2.y));
                                }
                            }
                            const float2 ri = ri2_mixed<KER>(r2, a.neg_kappa_log2e, SEL);
                            f[v] = fma2(sq, ri, f[v]);
                            g2 = fma2(qt[v], ri, g2);
                        }
                        gs[s8] = g2.x + g2.y;
                    }
                }
                const float wsum = warp_sum8(gs, lane);
                if ((lane & 3) == 0 && j8 + (lane >> 2) < je) sbuf[warp * kTile + j8 + (lane >> 2)] = wsum;
            }
#pragma unroll
            for (int v = 0; v < kH; ++v) {
                two_sum_add(hi[2 * v], lo[2 * v], f[v].x);
                two_sum_add(hi[2 * v + 1], lo[2 * v + 1], f[v].y);
            }
            if (CHECK && __any_sync(0xffffffffu, rmin < tau2)) {
                // Close pairs (see near_mixed), recomputed from FP64 coordinates for both
                // sides; the warp takes this branch together so the source-side corrections
                // can be added across lanes in a fixed order.
                for (int j = jb; j < je; ++j) {
                    const float4 p0 = sm[2 * j], p1 = sm[2 * j + 1];
                    const int ps = cs + j0 + j;
                    float cj = 0.f;
#pragma unroll
                    for (int u = 0; u < kT; ++u) {
                        const float2 ptx = tg.x[u / 2], pty = tg.y[u / 2], ptz = tg.z[u / 2];
                        const float dx = p0.x + ((u & 1) ? ptx.y : ptx.x);
                        const float dy = p0.z + ((u & 1) ? pty.y : pty.x);
                        const float dz = p1.x + ((u & 1) ? ptz.y : ptz.x);
                        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        if (r2 > 0.f && r2 < tau2) {
                            const int t = min(t0 + l + tpg * u, nb - 1);
                            const double ex = a.sx[ps] - a.tx[tb + t], ey = a.sy[ps] - a.ty[tb + t];
                            const double ez = a.sz[ps] - a.tz[tb + t];
                            const double r2d = ex * ex + ey * ey + ez * ez;
                            double rid = rsqrt(r2d);
                            if (KER == BLTC_KERNEL_YUKAWA) rid *= exp(-a.kappa * (r2d * rid));
                            float ri = rsqrt_approx(r2);
                            if (KER == BLTC_KERNEL_YUKAWA) ri *= ex2_approx(a.neg_kappa_log2e * (r2 * ri));
                            lo[u] += static_cast<float>(a.sq[ps] * rid - static_cast<double>(p1.z * ri));
                            const float qu = (u & 1) ? qt[u / 2].y : qt[u / 2].x;
                            if (qu != 0.f)
                                cj += static_cast<float>(a.sq[tb + t] * rid - static_cast<double>(qu * ri));
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) cj += __shfl_xor_sync(0xffffffffu, cj, o);
                    if (lane == 0) sbuf[warp * kTile + j] += cj;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kT; ++u) acc[u * kThreads] += static_cast<double>(hi[u]) + static_cast<double>(lo[u]);
        // C's row: each staged source's sum over the group's warps, in warp order
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += kThreads) {
            const int w0 = ((j / kBlock) % G) * wpg;
            double sum = 0.0;
            for (int w = w0; w < w0 + wpg; ++w) sum += static_cast<double>(sbuf[w * kTile + j]);
            if (t0 == 0) mrow[j0 + j] = sum; else mrow[j0 + j] += sum;
        }
    }
}

// Far field (Eq. 11) of cluster C on its tensor grid of Chebyshev points (Eq. 8).  Shared
// memory holds (s, s) pairs of the 3(n+1) point coordinates relative to the batch centre,
// then (qhat, qhat) pairs of the (n+1)^3 modified charges.  Within a (k1, k2) row the
// partial r^2 of a target is reused over the n+1 values of k3; runs of rows holding about
// kBlock terms are summed in FP32 and folded into a TwoSum accumulator.
template <int KER>
__device__ void far_mixed(const SweepArgs& a, int C, const double cb[3], const Targets& tg,
                          double* acc, float2* sm, int g, int G) {
    const int np1 = a.np1, n = np1 - 1, P = np1 * np1 * np1;
    const float* qh = a.qhat32 + static_cast<int64_t>(a.qslot[C]) * P;
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * np1; k += kThreads) {
        const int d = k / np1, kk = k - d * np1;
        const double s = cheb_point(a.cheb_t, kk, n, a.s_lo[3 * C + d], a.s_hi[3 * C + d]);
        const float v = __double2float_rn(s - (d == 0 ? cb[0] : (d == 1 ? cb[1] : cb[2])));
        sm[k] = make_float2(v, v);
    }
    float2* sq = sm + 3 * np1;
    for (int k = threadIdx.x; k < P; k += kThreads) {
        const float v = qh[k];
        sq[k] = make_float2(v, v);
    }
    __syncthreads();
    const float2* sxp = sm;
    const float2* syp = sm + np1;
    const float2* szp = sm + 2 * np1;
    float hi[kT], lo[kT];
#pragma unroll
    for (int u = 0; u < kT; ++u) hi[u] = lo[u] = 0.f;
    // rows are summed in FP32 in runs of about kBlock terms, then folded by TwoSum
    const int R = np1 * np1, run = max(1, kBlock / np1) * G;
    for (int row0 = g; row0 < R; row0 += run) {
        float2 f[kH];
#pragma unroll
        for (int v = 0; v < kH; ++v) f[v] = make_float2(0.f, 0.f);
        for (int row = row0; row < min(R, row0 + run); row += G) {
            const int k1 = row / np1, k2 = row - k1 * np1;
            const float2 sx = sxp[k1], sy = syp[k2];
            float2 t[kH];
#pragma unroll
            for (int v = 0; v < kH; ++v) {
                const float2 dx = add2(sx, tg.x[v]);
                const float2 dy = add2(sy, tg.y[v]);
                t[v] = fma2(dy, dy, mul2(dx, dx));
            }
            const float2* qrow = sq + row * np1;
#pragma unroll 9
            for (int k3 = 0; k3 < np1; ++k3) {
                const float2 sz = szp[k3], q = qrow[k3];
#pragma unroll
                for (int v = 0; v < kH; ++v) {
                    const float2 dz = add2(sz, tg.z[v]);
                    const float2 r2 = fma2(dz, dz, t[v]);
                    f[v] = fma2(q, ri2_mixed<KER>(r2, a.neg_kappa_log2e, false), f[v]);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < kH; ++v) {
            two_sum_add(hi[2 * v], lo[2 * v], f[v].x);
            two_sum_add(hi[2 * v + 1], lo[2 * v + 1], f[v].y);
        }
    }
#pragma unroll
    for (int u = 0; u < kT; ++u) acc[u * kThreads] += static_cast<double>(hi[u]) + static_cast<double>(lo[u]);
}

template <int KER>
__device__ void item_mixed(const SweepArgs& a, int4 it, float4* sm) {
    const int b = it.x;
    const int B = a.b_leaves[b];
    const int tb = a.b_begin[B], nb = a.b_count[B];
    const double cb[3] = {a.b_center[3 * B], a.b_center[3 * B + 1], a.b_center[3 * B + 2]};
    const int a0 = a.app_off[b], na = a.app_off[b + 1] - a0, d0 = a.dir_off[b];
    double* out = a.partials + a.part_off[b] + static_cast<int64_t>(it.w) * nb;
    const int G = groups_for(nb);
    const int tpg = kThreads / G;                       // threads per group
    const int g = static_cast<int>(threadIdx.x) / tpg, l = static_cast<int>(threadIdx.x) - g * tpg;
    for (int t0 = 0; t0 < nb; t0 += tpg * kT) {
        Targets tg;
        double* acc = reinterpret_cast<double*>(reinterpret_cast<char*>(sm) + kSmemBytes) + threadIdx.x;  // [u * kThreads]
#pragma unroll
        for (int u = 0; u < kT; ++u) {
            const int t = min(t0 + l + tpg * u, nb - 1);
            const float nx = -__double2float_rn(a.tx[tb + t] - cb[0]);
            const float ny = -__double2float_rn(a.ty[tb + t] - cb[1]);
            const float nz = -__double2float_rn(a.tz[tb + t] - cb[2]);
            if (u & 1) {
                tg.x[u / 2].y = nx;
                tg.y[u / 2].y = ny;
                tg.z[u / 2].y = nz;
            } else {
                tg.x[u / 2].x = nx;
                tg.y[u / 2].x = ny;
                tg.z[u / 2].x = nz;
            }
            acc[u * kThreads] = 0.0;
        }
        for (int e = it.y; e < it.z; ++e) {
            if (e < na)
                far_mixed<KER>(a, a.app_ids[a0 + e], cb, tg, acc, reinterpret_cast<float2*>(sm), g, G);
            else {
                const int de = d0 + e - na;
                const int C = a.dir_ids[de];
                const float tau2 = a.dir_tau2[de];
                const uint8_t sel = a.dir_sel[de];
                if (sel & kSelSkip) continue;            // evaluated by the partner's mutual entry
                if (sel & kSelMutual) {
                    float* sbuf = reinterpret_cast<float*>(reinterpret_cast<char*>(sm) + kSmemBytes + kAccBytes);
                    double* mrow = a.mpart + a.dir_moff[de];
                    switch (sel & (kSelZero | kSelClose)) {
                        case 0: near_mutual<KER, false, false>(a, C, tau2, cb, tg, acc, sm, sbuf, mrow, g, G, tb, nb, t0, l, tpg); break;
                        case kSelClose: near_mutual<KER, false, true>(a, C, tau2, cb, tg, acc, sm, sbuf, mrow, g, G, tb, nb, t0, l, tpg); break;
                        default: near_mutual<KER, true, true>(a, C, tau2, cb, tg, acc, sm, sbuf, mrow, g, G, tb, nb, t0, l, tpg); break;
                    }
                    continue;
                }
                switch (sel & (kSelZero | kSelClose)) {
                    case 0: near_mixed<KER, false, false>(a, C, tau2, cb, tg, acc, sm, g, G, tb, nb, t0, l, tpg); break;
                    case kSelClose: near_mixed<KER, false, true>(a, C, tau2, cb, tg, acc, sm, g, G, tb, nb, t0, l, tpg); break;
                    default: near_mixed<KER, true, true>(a, C, tau2, cb, tg, acc, sm, g, G, tb, nb, t0, l, tpg); break;
                }
            }
        }
        if (G == 1) {
#pragma unroll
            for (int u = 0; u < kT; ++u) {
                const int t = t0 + l + tpg * u;
                if (t < nb) out[t] = acc[u * kThreads];
            }
        } else {
            // add the groups' partials in group order
            double* red = reinterpret_cast<double*>(sm);   // [G][tpg * kT]
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kT; ++u) red[g * tpg * kT + u * tpg + l] = acc[u * kThreads];
            __syncthreads();
            for (int i = threadIdx.x; i < tpg * kT; i += kThreads) {
                double s2 = red[i];
                for (int gg = 1; gg < G; ++gg) s2 += red[gg * tpg * kT + i];
                const int u = i / tpg, t = t0 + (i - u * tpg) + tpg * u;
                if (t < nb) out[t] = s2;
            }
        }
    }
}

template <int KER>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_sweep_mixed(SweepArgs a) {
    extern __shared__ __align__(16) float4 sm_dyn[];
    float4* sm = sm_dyn;
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(a.counter, 1u));
        __syncthreads();
        const int i = s_item;
        if (i >= a.n_items) return;
        item_mixed<KER>(a, a.items[i], sm);
    }
}

// Several requests' sweeps in one persistent launch (the serving engine).  `order` lists
// (request, item) pairs longest first; each block copies the request's arguments to shared
// memory when the request changes.  An item computes exactly what it computes in a
// single-request launch, so every request's potentials are the same bits alone or in a mix.
template <int KER>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_sweep_multi(const SweepArgs* __restrict__ reqs,
                                                             const int2* __restrict__ order,
                                                             int total, unsigned int* counter) {
    extern __shared__ __align__(16) float4 sm_dyn[];
    float4* sm = sm_dyn;
    __shared__ __align__(16) SweepArgs s_a;
    __shared__ int s_item;
    int cur = -1;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(counter, 1u));
        __syncthreads();
        const int i = s_item;
        if (i >= total) return;
        const int2 o = order[i];
        if (o.x != cur) {
            const int* src = reinterpret_cast<const int*>(reqs + o.x);
            int* dst = reinterpret_cast<int*>(&s_a);
            for (int w = threadIdx.x; w < static_cast<int>(sizeof(SweepArgs) / sizeof(int)); w += kThreads) dst[w] = src[w];
            cur = o.x;
            __syncthreads();
        }
        item_mixed<KER>(s_a, s_a.items[o.y], sm);
    }
}

// ---- FP64 ---------------------------------------------------------------------------

template <int KER>
__device__ __forceinline__ double g_fp64(double r2, double q, double kappa) {
    double ri = rsqrt(r2);
    if (KER == BLTC_KERNEL_YUKAWA) ri *= exp(-kappa * (r2 * ri));
    return q * ri;
}

template <int KER, int T>
__device__ void near_fp64(const SweepArgs& a, int C, const double (&xt)[T], const double (&yt)[T],
                          const double (&zt)[T], double (&acc)[T], D4* sm) {
    const int cs = a.s_begin[C], nc = a.s_count[C];
    for (int j0 = 0; j0 < nc; j0 += kSrcTile64) {
        const int m = min(kSrcTile64, nc - j0);
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += kThreads) {
            const int p = cs + j0 + j;
            sm[j] = D4{a.sx[p], a.sy[p], a.sz[p], a.sq[p]};
        }
        __syncthreads();
        for (int j = 0; j < m; ++j) {
            const D4 s = sm[j];
#pragma unroll
            for (int u = 0; u < T; ++u) {
                const double dx = xt[u] - s.x, dy = yt[u] - s.y, dz = zt[u] - s.z;
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 != 0.0) acc[u] += g_fp64<KER>(r2, s.w, a.kappa);
            }
        }
    }
}

template <int KER, int T>
__device__ void far_fp64(const SweepArgs& a, int C, const double (&xt)[T], const double (&yt)[T],
                         const double (&zt)[T], double (&acc)[T], double* sm) {
    const int np1 = a.np1, n = np1 - 1, P = np1 * np1 * np1;
    const double* qh = a.qhat64 + static_cast<int64_t>(a.qslot[C]) * P;
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * np1; k += kThreads) {
        const int d = k / np1, kk = k - d * np1;
        sm[k] = cheb_point(a.cheb_t, kk, n, a.s_lo[3 * C + d], a.s_hi[3 * C + d]);
    }
    double* sq = sm + 3 * np1;
    for (int k = threadIdx.x; k < P; k += kThreads) sq[k] = qh[k];
    __syncthreads();
    for (int k1 = 0; k1 < np1; ++k1) {
        double dx2[T];
#pragma unroll
        for (int u = 0; u < T; ++u) {
            const double dx = xt[u] - sm[k1];
            dx2[u] = dx * dx;
        }
        for (int k2 = 0; k2 < np1; ++k2) {
            double t[T];
#pragma unroll
            for (int u = 0; u < T; ++u) {
                const double dy = yt[u] - sm[np1 + k2];
                t[u] = dx2[u] + dy * dy;
            }
            const double* qrow = sq + (k1 * np1 + k2) * np1;
            for (int k3 = 0; k3 < np1; ++k3) {
                const double q = qrow[k3], szk = sm[2 * np1 + k3];
#pragma unroll
                for (int u = 0; u < T; ++u) {
                    const double dz = zt[u] - szk;
                    acc[u] += g_fp64<KER>(t[u] + dz * dz, q, a.kappa);
                }
            }
        }
    }
}

template <int KER, int T>
__device__ void item_fp64(const SweepArgs& a, int4 it, D4* sm) {
    const int b = it.x;
    const int B = a.b_leaves[b];
    const int tb = a.b_begin[B], nb = a.b_count[B];
    const int a0 = a.app_off[b], na = a.app_off[b + 1] - a0, d0 = a.dir_off[b];
    double* out = a.partials + a.part_off[b] + static_cast<int64_t>(it.w) * nb;
    for (int t0 = 0; t0 < nb; t0 += kThreads * T) {
        double xt[T], yt[T], zt[T], acc[T];
#pragma unroll
        for (int u = 0; u < T; ++u) {
            const int t = min(t0 + static_cast<int>(threadIdx.x) + kThreads * u, nb - 1);
            xt[u] = a.tx[tb + t];
            yt[u] = a.ty[tb + t];
            zt[u] = a.tz[tb + t];
            acc[u] = 0.0;
        }
        for (int e = it.y; e < it.z; ++e) {
            if (e < na)
                far_fp64<KER, T>(a, a.app_ids[a0 + e], xt, yt, zt, acc, reinterpret_cast<double*>(sm));
            else
                near_fp64<KER, T>(a, a.dir_ids[d0 + e - na], xt, yt, zt, acc, sm);
        }
#pragma unroll
        for (int u = 0; u < T; ++u) {
            const int t = t0 + static_cast<int>(threadIdx.x) + kThreads * u;
            if (t < nb) out[t] = acc[u];
        }
    }
}

template <int KER>
__global__ void __launch_bounds__(kThreads, 2) k_sweep_fp64(SweepArgs a) {
    __shared__ __align__(16) D4 sm[kSmemBytes / sizeof(D4)];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(a.counter, 1u));
        __syncthreads();
        const int i = s_item;
        if (i >= a.n_items) return;
        const int4 it = a.items[i];
        const int nb = a.b_count[a.b_leaves[it.x]];
        if (nb <= kThreads)
            item_fp64<KER, 1>(a, it, sm);
        else if (nb <= 2 * kThreads)
            item_fp64<KER, 2>(a, it, sm);
        else
            item_fp64<KER, 4>(a, it, sm);
    }
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
};

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
    if (e >= n_dir) return;
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
    if (b < a.n_batches) lidx[a.b_leaves[b]] = static_cast<int32_t>(b);
}

__global__ void k_mutual_mark(PlanArgs a, int64_t n_dir) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= n_dir) return;
    const int64_t b = batch_of_entry(a, e);
    const int A = a.b_leaves[b], C = a.dir_ids[e];
    int32_t partner = -1;
    int64_t len = 0;
    const int b2 = C != A && a.s_nch[C] == 0 ? a.lidx[C] : -1;
    if (b2 >= 0) {
        int lo = a.dir_off[b2], hi = a.dir_off[b2 + 1];       // search A in [lo, hi)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (a.dir_ids[mid] < A) lo = mid + 1; else hi = mid;
        }
        if (lo < a.dir_off[b2 + 1] && a.dir_ids[lo] == A) {
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
    if (e >= n_dir) return;
    const uint8_t sel = a.dir_sel[e];
    a.dir_moff[e] = (sel & kSelMutual) ? a.moff_e[e] : ((sel & kSelSkip) ? a.moff_e[a.partner[e]] : -1);
}

__global__ void k_batch_cost(PlanArgs a) {
    const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= a.n_batches) return;
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
                             int64_t* cost) {
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

// Per target: its items' partials in item order, then (mutual pairs) the rows that partner
// batches wrote for it, in list order; scattered to the caller's order.  Each thread keeps 8
// targets so that every row is read with 8 independent, coalesced loads in flight.
__global__ void k_finalize(const int32_t* __restrict__ b_leaves, const int32_t* __restrict__ b_begin,
                           const int32_t* __restrict__ b_count, const int32_t* __restrict__ perm,
                           const int32_t* __restrict__ n_chunks, const int64_t* __restrict__ part_off,
                           const double* __restrict__ partials, const int32_t* __restrict__ dir_off,
                           const uint8_t* __restrict__ dir_sel, const int64_t* __restrict__ dir_moff,
                           const double* __restrict__ mpart, double* __restrict__ phi) {
    constexpr int U = 8;
    const int b = blockIdx.x;
    const int B = b_leaves[b];
    const int tb = b_begin[B], nb = b_count[B], K = n_chunks[b];
    const double* p = partials + part_off[b];
    for (int t0 = 0; t0 < nb; t0 += U * static_cast<int>(blockDim.x)) {
        double s[U];
#pragma unroll
        for (int u = 0; u < U; ++u) s[u] = 0.0;
        for (int c = 0; c < K; ++c) {
            const double* row = p + static_cast<int64_t>(c) * nb;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0 + static_cast<int>(threadIdx.x) + u * static_cast<int>(blockDim.x);
                if (t < nb) s[u] += row[t];
            }
        }
        if (mpart) {
            for (int e = dir_off[b]; e < dir_off[b + 1]; ++e) {
                if (!(dir_sel[e] & kSelSkip)) continue;
                const double* row = mpart + dir_moff[e];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int t = t0 + static_cast<int>(threadIdx.x) + u * static_cast<int>(blockDim.x);
                    if (t < nb) s[u] += row[t];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int t = t0 + static_cast<int>(threadIdx.x) + u * static_cast<int>(blockDim.x);
            if (t < nb) phi[perm[tb + t]] = s[u];
        }
    }
}

__global__ void k_counts(const int32_t* b_leaves, const int32_t* b_count, const int32_t* s_count,
                         const int32_t* app_off, const int32_t* dir_off, const int32_t* dir_ids,
                         const uint8_t* dir_sel, int64_t n_batches, int64_t P, unsigned long long* out) {
    const int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= n_batches) return;
    const int64_t nb = b_count[b_leaves[b]];
    int64_t d = 0, de = 0;
    for (int e = dir_off[b]; e < dir_off[b + 1]; ++e) {
        d += s_count[dir_ids[e]];
        if (!dir_sel || !(dir_sel[e] & kSelSkip)) de += s_count[dir_ids[e]];
    }
    atomicAdd(&out[0], static_cast<unsigned long long>(d * nb));
    atomicAdd(&out[1], static_cast<unsigned long long>(static_cast<int64_t>(app_off[b + 1] - app_off[b]) * P * nb));
    atomicAdd(&out[2], static_cast<unsigned long long>(de * nb));
}

}  // namespace

void build_plan(Context* ctx, Lists* L, int degree, bool mutual) {
    cudaStream_t s = ctx->stream;
    const int64_t nb = L->n_batches;
    const int64_t np1 = degree + 1;
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
    const int64_t* w0 = ctx->read_words(words.p, 4);
    const int64_t total = w0[0];
    if (pl.mutual) pl.mpart_len = w0[3];
    const int64_t blocks = kMinBlocks * static_cast<int64_t>(std::max(1, ctx->sm_count));
    a.cut = std::max<int64_t>(total / (blocks * kItemsPerBlock), int64_t(1) << 20);
    pl.n_chunks = DBuf<int32_t>(ctx, nb);
    pl.part_off = DBuf<int64_t>(ctx, nb);
    DBuf<int32_t> item_off(ctx, nb);
    a.n_chunks = pl.n_chunks.p;
    a.part_len = part_len.p;
    k_chunks<false><<<grid_for(nb, 128), 128, 0, s>>>(a); ++ctx->launches;
    BLTC_LAUNCH_CHECK("plan chunks");
    exclusive_scan_i32(ctx, pl.n_chunks.p, item_off.p, nb, reinterpret_cast<int32_t*>(words.p + 1));
    exclusive_scan_i64(ctx, part_len.p, pl.part_off.p, nb, words.p + 2);
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
        k_item_costs<<<grid_for(pl.n_items, 256), 256, 0, s>>>(a, pl.items.p, pl.n_items, icost.p); ++ctx->launches;
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
    const double kappa = p.kernel == BLTC_KERNEL_YUKAWA ? p.kappa : 0.0;
    a.kappa = kappa;
    a.neg_kappa_log2e = static_cast<float>(-kappa * 1.4426950408889634);
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
    cudaStream_t s = ctx->stream;
    prepare_plan(ctx, L, p.degree, p.precision);
    Plan& pl = L->plan;
    DBuf<double> partials(ctx, pl.partial_len);
    DBuf<double> mpart(ctx, pl.mutual ? pl.mpart_len : 0);
    DBuf<unsigned int> counter(ctx, 1);
    BLTC_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned int), s));
    SweepArgs a = make_args(ctx, L, bt, st, p, partials.p, counter.p);
    a.mpart = pl.mutual ? mpart.p : nullptr;
    const int per_sm = p.precision == BLTC_PRECISION_MIXED ? kMinBlocks : 2;
    const unsigned grid = static_cast<unsigned>(
        std::min<int64_t>(pl.n_items, per_sm * static_cast<int64_t>(std::max(1, ctx->sm_count))));
    ctx->mark(Context::kSweepBegin);
    if (pl.n_items > 0) {
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
        partials.p, L->dir_off.p, pl.dir_sel.p, a.dir_moff, a.mpart, phi); ++ctx->launches;
    BLTC_LAUNCH_CHECK("finalize");
    ctx->mark(Context::kEnd);
}

void evaluate_multi(Context* ctx, const std::vector<SweepJob>& jobs) {
    if (jobs.empty()) return;
    cudaStream_t s = ctx->stream;
    const int R = static_cast<int>(jobs.size());
    std::vector<DBuf<double>> partials, mparts;
    std::vector<SweepArgs> args;
    partials.reserve(jobs.size());
    mparts.reserve(jobs.size());
    args.reserve(jobs.size());
    DBuf<unsigned int> counter(ctx, 1);
    BLTC_CUDA(cudaMemsetAsync(counter.p, 0, sizeof(unsigned int), s));
    // global longest-first order over all requests' items
    std::vector<std::pair<int64_t, int2>> all;
    for (int r = 0; r < R; ++r) {
        const SweepJob& j = jobs[static_cast<size_t>(r)];
        require(j.p.precision == BLTC_PRECISION_MIXED, "serving runs the mixed-precision sweep");
        check_eval(j.L, j.bt, j.st, j.p, j.phi);
        if (!j.L->plan.valid || j.L->plan.degree != j.p.degree ||
            j.L->plan.mutual != (j.L->bt == j.L->st && j.L->n_dir > 0))
            throw Error(BLTC_ERR_STATE, "evaluate_multi: request has no work plan");
        const Plan& pl = j.L->plan;
        partials.emplace_back(ctx, pl.partial_len);
        mparts.emplace_back(ctx, pl.mutual ? pl.mpart_len : 0);
        args.push_back(make_args(ctx, j.L, j.bt, j.st, j.p, partials.back().p, counter.p));
        args.back().mpart = pl.mutual ? mparts.back().p : nullptr;
        for (int64_t i = 0; i < pl.n_items; ++i)
            all.push_back({pl.h_cost[static_cast<size_t>(i)], make_int2(r, static_cast<int>(i))});
    }
    std::stable_sort(all.begin(), all.end(), [](const std::pair<int64_t, int2>& x,
                                                const std::pair<int64_t, int2>& y) { return x.first > y.first; });
    // one persistent launch per kernel type present (each instantiation keeps its registers)
    std::vector<int2> order[2];
    for (const auto& pr : all) order[jobs[static_cast<size_t>(pr.second.x)].p.kernel == BLTC_KERNEL_YUKAWA].push_back(pr.second);
    DBuf<SweepArgs> d_args(ctx, R);
    DBuf<int2> d_order(ctx, static_cast<int64_t>(all.size()));
    DBuf<unsigned int> counter2(ctx, 1);
    BLTC_CUDA(cudaMemsetAsync(counter2.p, 0, sizeof(unsigned int), s));
    BLTC_CUDA(cudaMemcpyAsync(d_args.p, args.data(), sizeof(SweepArgs) * R, cudaMemcpyHostToDevice, s));
    if (!order[0].empty())
        BLTC_CUDA(cudaMemcpyAsync(d_order.p, order[0].data(), sizeof(int2) * order[0].size(), cudaMemcpyHostToDevice, s));
    if (!order[1].empty())
        BLTC_CUDA(cudaMemcpyAsync(d_order.p + order[0].size(), order[1].data(), sizeof(int2) * order[1].size(),
                                  cudaMemcpyHostToDevice, s));
    // the host vectors must outlive the asynchronous copies
    BLTC_CUDA(cudaStreamSynchronize(s));
    const int64_t cap = kMinBlocks * static_cast<int64_t>(std::max(1, ctx->sm_count));
    if (!order[0].empty()) {
        const int total = static_cast<int>(order[0].size());
        BLTC_CUDA(cudaFuncSetAttribute(k_sweep_multi<BLTC_KERNEL_COULOMB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmem));
        k_sweep_multi<BLTC_KERNEL_COULOMB><<<static_cast<unsigned>(std::min<int64_t>(total, cap)), kThreads, kMixedSmem, s>>>(
            d_args.p, d_order.p, total, counter.p); ++ctx->launches;
        BLTC_LAUNCH_CHECK("sweep multi coulomb");
    }
    if (!order[1].empty()) {
        const int total = static_cast<int>(order[1].size());
        BLTC_CUDA(cudaFuncSetAttribute(k_sweep_multi<BLTC_KERNEL_YUKAWA>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kMixedSmem));
        k_sweep_multi<BLTC_KERNEL_YUKAWA><<<static_cast<unsigned>(std::min<int64_t>(total, cap)), kThreads, kMixedSmem, s>>>(
            d_args.p, d_order.p + order[0].size(), total, counter2.p); ++ctx->launches;
        BLTC_LAUNCH_CHECK("sweep multi yukawa");
    }
    for (int r = 0; r < R; ++r) {
        const SweepJob& j = jobs[static_cast<size_t>(r)];
        const Plan& pl = j.L->plan;
        k_finalize<<<static_cast<unsigned>(j.L->n_batches), 256, 0, s>>>(
            j.bt->leaves.p, j.bt->begin.p, j.bt->count.p, j.bt->perm.p, pl.n_chunks.p, pl.part_off.p,
            partials[static_cast<size_t>(r)].p, j.L->dir_off.p, pl.dir_sel.p,
            pl.mutual ? pl.dir_moff.p : nullptr, pl.mutual ? mparts[static_cast<size_t>(r)].p : nullptr,
            j.phi); ++ctx->launches;
        BLTC_LAUNCH_CHECK("finalize multi");
    }
}

static void counts(Context* ctx, const Lists* L, const uint8_t* dir_sel, int64_t* out3) {
    DBuf<int64_t> w(ctx, 3);
    BLTC_CUDA(cudaMemsetAsync(w.p, 0, 3 * sizeof(int64_t), ctx->stream));
    const int64_t np1 = L->degree + 1;
    k_counts<<<grid_for(L->n_batches, 128), 128, 0, ctx->stream>>>(
        L->bt->leaves.p, L->bt->count.p, L->st->count.p, L->app_off.p, L->dir_off.p,
        L->dir_ids.p, dir_sel, L->n_batches, np1 * np1 * np1, reinterpret_cast<unsigned long long*>(w.p)); ++ctx->launches;
    BLTC_LAUNCH_CHECK("counts");
    const int64_t* r = ctx->read_words(w.p, 3);
    for (int i = 0; i < 3; ++i) out3[i] = r[i];
}

void interaction_counts(Context* ctx, const Lists* L, int64_t* n_dir, int64_t* n_app) {
    int64_t r[3];
    counts(ctx, L, nullptr, r);
    if (n_dir) *n_dir = r[0];
    if (n_app) *n_app = r[1];
}

int64_t plan_evaluations(Context* ctx, Lists* L, int degree, int precision) {
    require(degree == L->degree, "evaluations: the lists were built for another degree");
    prepare_plan(ctx, L, degree, precision);
    int64_t r[3];
    counts(ctx, L, L->plan.dir_sel.p, r);
    return r[1] + r[2];
}

}  // namespace bltc
