// sweep_device.cuh -- device code of the far- and near-field sweeps (A3, A4).
//
// Shared by the compiled library (sweep.cu) and by run-time compilation of user kernels
// (user_kernel.cu compiles this text with NVRTC, with BLTC_NVRTC defined and the functions
// bltc_user_g32 / bltc_user_g64 supplied by the user).  Nothing here may include a host
// header when BLTC_NVRTC is defined.
#pragma once
#ifndef BLTC_NVRTC
#include <cstdint>

#include "bltc.h"
#include "internal.cuh"
#endif

namespace bltc {
namespace sweepdev {

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
    const double *b_lo, *b_hi;         // batch boxes (close-pair screening)
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
    float* mpart;              // mutual rows (FP32): potentials a batch's particles induce on a partner's
    const int4* items;
    const int64_t* part_off;
    double* partials;
    int n_items;
    unsigned int* counter;
    // kernel
    int kernel;
    double kappa;
    float neg_kappa_log2e;
    float param32;             // kappa in FP32, the parameter of a user kernel
    int g_max;                 // cap on the source groups of a batch (1, 2, 4 or 8)
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

// ---- kernels G(r) ----------------------------------------------------------------------

// Template value of a user kernel (bltc_kernel_register): its G comes from the functions
// bltc_user_g32 / bltc_user_g64, which exist only in the run-time compiled module.
constexpr int kKerUser = 2;

// G(r) without the charge for one pair with r^2 = r2 > 0, FP32: 1/r, or e^{-kappa r}/r as
// 2^{-kappa log2(e) r} / r (Eq. 2).  The charge multiplies last, so kappa = 0 reproduces
// Coulomb bit for bit.
template <int KER>
__device__ __forceinline__ float g32(float r2, float nkl2e, float param) {
    float ri = rsqrt_approx(r2);
#ifdef BLTC_NVRTC
    if constexpr (KER == kKerUser) return bltc_user_g32(r2, r2 * ri, param);
#endif
    if (KER == BLTC_KERNEL_YUKAWA) ri *= ex2_approx(nkl2e * (r2 * ri));
    return ri;
}

// The same in FP64.
template <int KER>
__device__ __forceinline__ double g64(double r2, double kappa) {
#ifdef BLTC_NVRTC
    if constexpr (KER == kKerUser) return bltc_user_g64(r2, sqrt(r2), kappa);
#endif
    double ri = rsqrt(r2);
    if (KER == BLTC_KERNEL_YUKAWA) ri *= exp(-kappa * (r2 * ri));
    return ri;
}

// ---- mixed precision ------------------------------------------------------------------

// Packed FP32x2 arithmetic (FADD2 / FMUL2 / FFMA2 on sm_100 and later): one instruction
// works on two targets, which halves the FMA-pipe issue slots per interaction so that the
// SFU (one MUFU.RSQ per interaction) becomes the binding pipe.  Each lane of a packed
// operation rounds exactly like the scalar operation, so both paths give identical bits.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// G without the charge for two pairs (packed), zero where skip_zero and r^2 == 0.
template <int KER>
__device__ __forceinline__ float2 ri2_mixed(float2 r2, float nkl2e, float param, bool skip_zero) {
    if constexpr (KER == kKerUser) {
        float2 g = make_float2(r2.x > 0.f ? g32<KER>(r2.x, nkl2e, param) : 0.f,
                               r2.y > 0.f ? g32<KER>(r2.y, nkl2e, param) : 0.f);
        return g;
    }
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
// of 256/G threads (G = 1, 2, 4 or 8): every group covers all targets of the batch, in passes
// of 2048/G targets, and takes every G-th block of work of each cluster (blocks of kBlock
// sources in the near field, (k1, k2) rows of the proxy grid in the far field).  Each group
// keeps its own partial potentials; they are added in group order at the end of the item, so
// the result is fixed by the batch alone.  The last pass runs its padding slots like targets,
// so G is the one with the fewest target slots, ceil(nb / (2048/G)) * 2048/G, the smallest G
// on a tie, up to the tile's cap g_max: a batch of 1100 targets runs 1280 slots with G = 8
// instead of 2048 with G = 1.
__device__ __forceinline__ int groups_for(int nb, int g_max) {
    int best = 1, best_slots = (nb + kThreads * kT - 1) / (kThreads * kT) * (kThreads * kT);
#pragma unroll
    for (int G = 2; G <= 8; G *= 2) {
        if (G > g_max) break;
        const int w = kThreads / G * kT;
        const int slots = (nb + w - 1) / w * w;
        if (slots < best_slots) {
            best = G;
            best_slots = slots;
        }
    }
    return best;
}

// Close-pair screening per block of kBlock staged sources.  A source farther than tau from the
// batch box is farther than tau from every target, so a block of such sources needs no
// running minimum of r^2.  The test runs on the FP32 batch-relative coordinates with the
// distance doubled (4 tau^2), far above their rounding (about 2^-24 of the box extent).
constexpr bool kCloseBlockScreen = true;

// Batch box relative to the batch centre, FP32: lo in .x/.y/.z of bl, hi in bh.
__device__ __forceinline__ void batch_box_rel(const SweepArgs& a, int B, const double cb[3], float3& bl, float3& bh) {
    bl = make_float3(__double2float_rn(a.b_lo[3 * B] - cb[0]), __double2float_rn(a.b_lo[3 * B + 1] - cb[1]),
                     __double2float_rn(a.b_lo[3 * B + 2] - cb[2]));
    bh = make_float3(__double2float_rn(a.b_hi[3 * B] - cb[0]), __double2float_rn(a.b_hi[3 * B + 1] - cb[1]),
                     __double2float_rn(a.b_hi[3 * B + 2] - cb[2]));
}

// Stages sources [j0, j0 + m) of cluster C as (x, x, y, y), (z, z, q, q) relative to the batch
// centre; with SCREEN, blk[b] = 1 when block b of kBlock staged sources holds a source within
// 2 tau of the batch box.  Every thread of the block calls it (the flags are warp votes).
template <bool SCREEN>
__device__ __forceinline__ void stage_near(const SweepArgs& a, int p0, int m, const double cb[3], float4* sm,
                                           uint8_t* blk, float3 bl, float3 bh, float tau2) {
    for (int j0 = 0; j0 < m; j0 += kThreads) {
        const int j = j0 + static_cast<int>(threadIdx.x);
        bool close = false;
        if (j < m) {
            const int p = p0 + j;
            const float sx = __double2float_rn(a.sx[p] - cb[0]);
            const float sy = __double2float_rn(a.sy[p] - cb[1]);
            const float sz = __double2float_rn(a.sz[p] - cb[2]);
            const float sq = __double2float_rn(a.sq[p]);
            sm[2 * j] = make_float4(sx, sx, sy, sy);
            sm[2 * j + 1] = make_float4(sz, sz, sq, sq);
            if (SCREEN) {
                const float gx = fmaxf(fmaxf(bl.x - sx, sx - bh.x), 0.f);
                const float gy = fmaxf(fmaxf(bl.y - sy, sy - bh.y), 0.f);
                const float gz = fmaxf(fmaxf(bl.z - sz, sz - bh.z), 0.f);
                close = fmaf(gx, gx, fmaf(gy, gy, gz * gz)) < 4.f * tau2;
            }
        }
        if (SCREEN) {
            static_assert(kBlock == 32, "one warp vote per block of staged sources");
            const unsigned v = __ballot_sync(0xffffffffu, close);
            const int first = j0 + (static_cast<int>(threadIdx.x) & ~31);
            if ((threadIdx.x & 31) == 0 && first < m) blk[first / kBlock] = v != 0u;
        }
    }
}

// One block [jb, je) of staged sources against this thread's targets: packed FP32 sums in f,
// and with CHK the smallest non-zero r^2 met, for the close-pair correction.
template <int KER, bool SEL, bool CHK>
__device__ __forceinline__ void near_block(const SweepArgs& a, const float4* sm, int jb, int je, const Targets& tg,
                                           float2 (&f)[kH], float& rmin) {
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
            if (CHK) {
                if (SEL) {
                    rmin = fminf(rmin, r2.x > 0.f ? r2.x : 3.0e38f);
                    rmin = fminf(rmin, r2.y > 0.f ? r2.y : 3.0e38f);
                } else {
                    rmin = fminf(rmin, fminf(r2.x, r2.y));
                }
            }
            f[v] = fma2(sq, ri2_mixed<KER>(r2, a.neg_kappa_log2e, a.param32, SEL), f[v]);
        }
    }
}

// Near field (Eq. 9) of cluster C.  Shared memory holds each staged source as two float4:
// (x, x, y, y) and (z, z, q, q), relative to the batch centre, so a packed operand is one
// aligned register pair.  Sums run over blocks of kBlock sources in FP32, folded into a
// TwoSum accumulator, then into FP64 per staged tile.
template <int KER, bool SEL, bool CHECK>
__device__ void near_mixed(const SweepArgs& a, int C, int B, float tau2, const double cb[3], const Targets& tg,
                           double* acc, float4* sm, int g, int G, int tb, int nb, int t0,
                           int l, int tpg) {
    constexpr int kTile = kNearTile;
    constexpr bool SCREEN = CHECK && kCloseBlockScreen;
    __shared__ uint8_t blk[kTile / kBlock];
    const int cs = a.s_begin[C], nc = a.s_count[C];
    float3 bl = make_float3(0.f, 0.f, 0.f), bh = bl;
    if (SCREEN) batch_box_rel(a, B, cb, bl, bh);
    for (int j0 = 0; j0 < nc; j0 += kTile) {
        const int m = min(kTile, nc - j0);
        __syncthreads();
        stage_near<SCREEN>(a, cs + j0, m, cb, sm, blk, bl, bh, tau2);
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
            if (CHECK && (!SCREEN || blk[jb / kBlock]))
                near_block<KER, SEL, CHECK>(a, sm, jb, je, tg, f, rmin);
            else
                near_block<KER, SEL, false>(a, sm, jb, je, tg, f, rmin);
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
                            const double rid = g64<KER>(r2d, a.kappa);
                            const float ri = g32<KER>(r2, a.neg_kappa_log2e, a.param32);
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

// Eight staged sources [j8, j8 + 8) of a mutual pair (with GUARD, those below je): this
// thread's packed sums in f, each source's sum over the warp's targets into sbuf.  Full groups
// run without the per-source bound test, which otherwise costs more than 6% of the sweep.
template <int KER, bool SEL, bool CHK, bool GUARD>
__device__ __forceinline__ void near_mutual_group(const SweepArgs& a, const float4* sm, int j8, int je,
                                                  const Targets& tg, const float2 (&qt)[kH], float2 (&f)[kH],
                                                  float& rmin, float* sbuf, int warp, int lane) {
    constexpr int kTile = kNearTile;
        float gs[8];
#pragma unroll
        for (int s8 = 0; s8 < 8; ++s8) {
            gs[s8] = 0.f;
            if (!GUARD || j8 + s8 < je) {
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
                    if (CHK) {
                        if (SEL) {
                            rmin = fminf(rmin, r2.x > 0.f ? r2.x : 3.0e38f);
                            rmin = fminf(rmin, r2.y > 0.f ? r2.y : 3.0e38f);
                        } else {
                            rmin = fminf(rmin, fminf(r2.x, r2.y));
                        }
                    }
                    const float2 ri = ri2_mixed<KER>(r2, a.neg_kappa_log2e, a.param32, SEL);
                    f[v] = fma2(sq, ri, f[v]);
                    g2 = fma2(qt[v], ri, g2);
                }
                gs[s8] = g2.x + g2.y;
            }
        }
        const float wsum = warp_sum8(gs, lane);
        if ((lane & 3) == 0 && (!GUARD || j8 + (lane >> 2) < je)) sbuf[warp * kTile + j8 + (lane >> 2)] = wsum;
}

// One block [jb, je) of staged sources of a mutual pair: packed sums for this thread's targets
// in f, each source's sum over the warp's targets into sbuf, and with CHK the smallest
// non-zero r^2 met.
template <int KER, bool SEL, bool CHK>
__device__ __forceinline__ void near_mutual_block(const SweepArgs& a, const float4* sm, int jb, int je,
                                                  const Targets& tg, const float2 (&qt)[kH], float2 (&f)[kH],
                                                  float& rmin, float* sbuf, int warp, int lane) {
    const int jfull = jb + ((je - jb) & ~7);
    int j8 = jb;
    for (; j8 < jfull; j8 += 8) near_mutual_group<KER, SEL, CHK, false>(a, sm, j8, je, tg, qt, f, rmin, sbuf, warp, lane);
    if (j8 < je) near_mutual_group<KER, SEL, CHK, true>(a, sm, j8, je, tg, qt, f, rmin, sbuf, warp, lane);
}

// Near field of a mutual pair: batch B (the targets) and leaf C are each in the other's
// direct list and are the same particles as sources and targets, so one evaluation of
// G(x_i, y_j) serves both phi_i += G q_j (as in near_mixed) and phi_j += G q_i (Eq. 9 for C's
// own batch, whose list entry for B is skipped).  The second sum runs over B's targets,
// which sit in different lanes: per source, each lane adds its 8 targets' q_i G in FP32, the
// warp adds its lanes (warp_sum8), and after the tile the group's warps are added in warp
// order into C's mutual row (FP32), so the result does not depend on scheduling.
template <int KER, bool SEL, bool CHECK>
__device__ void near_mutual(const SweepArgs& a, int C, int B, float tau2, const double cb[3], const Targets& tg,
                            double* acc, float4* sm, float* sbuf, float* mrow, int g, int G, int tb,
                            int nb, int t0, int l, int tpg) {
    constexpr int kTile = kNearTile;
    constexpr bool SCREEN = CHECK && kCloseBlockScreen;
    __shared__ uint8_t blk[kTile / kBlock];
    const int cs = a.s_begin[C], nc = a.s_count[C];
    float3 bl = make_float3(0.f, 0.f, 0.f), bh = bl;
    if (SCREEN) batch_box_rel(a, B, cb, bl, bh);
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
        stage_near<SCREEN>(a, cs + j0, m, cb, sm, blk, bl, bh, tau2);
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
            if (CHECK && (!SCREEN || blk[jb / kBlock]))
                near_mutual_block<KER, SEL, CHECK>(a, sm, jb, je, tg, qt, f, rmin, sbuf, warp, lane);
            else
                near_mutual_block<KER, SEL, false>(a, sm, jb, je, tg, qt, f, rmin, sbuf, warp, lane);
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
                            const double rid = g64<KER>(r2d, a.kappa);
                            const float ri = g32<KER>(r2, a.neg_kappa_log2e, a.param32);
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
            float hs = 0.f, ls = 0.f;       // TwoSum pair: about twice the FP32 precision
            for (int w = w0; w < w0 + wpg; ++w) two_sum_add(hs, ls, sbuf[w * kTile + j]);
            const float sum = hs + ls;
            if (t0 == 0) mrow[j0 + j] = sum; else mrow[j0 + j] += sum;
        }
    }
}

// Far field (Eq. 11) of cluster C on its tensor grid of Chebyshev points (Eq. 8).  Shared
// memory holds (s, s) pairs of the 3(n+1) point coordinates relative to the batch centre,
// then (qhat, qhat) pairs of the (n+1)^3 modified charges.  Within a (k1, k2) row the
// partial r^2 of a target is reused over the n+1 values of k3; runs of rows holding about
// kBlock terms are summed in FP32 and folded into the caller's TwoSum accumulator (hi, lo),
// which spans all far-field clusters of the work item and is converted to FP64 once: FP64
// adds run at a small fraction of the FP32 rate on this GPU.
template <int KER>
__device__ void far_mixed(const SweepArgs& a, int C, const double cb[3], const Targets& tg,
                          float (&hi)[kT], float (&lo)[kT], float2* sm, int g, int G) {
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
    // rows are summed in FP32 in runs of about kBlock terms, then folded by TwoSum
    const int R = np1 * np1, run = max(1, kBlock / np1) * G;
    int k1 = g / np1, k2 = g - k1 * np1;          // (k1, k2) of the current row, stepped by G
    for (int row0 = g; row0 < R; row0 += run) {
        float2 f[kH];
#pragma unroll
        for (int v = 0; v < kH; ++v) f[v] = make_float2(0.f, 0.f);
        for (int row = row0; row < min(R, row0 + run); row += G) {
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
                    f[v] = fma2(q, ri2_mixed<KER>(r2, a.neg_kappa_log2e, a.param32, false), f[v]);
                }
            }
            for (k2 += G; k2 >= np1; k2 -= np1) ++k1;
        }
#pragma unroll
        for (int v = 0; v < kH; ++v) {
            two_sum_add(hi[2 * v], lo[2 * v], f[v].x);
            two_sum_add(hi[2 * v + 1], lo[2 * v + 1], f[v].y);
        }
    }
}

// Far field of cluster C with barycentric Hermite charges, mixed precision.  With e = s - x
// (the source point minus the target, batch-relative FP32) the mixed derivatives are
// D^a G = (-1)^|a| prod_{a_l = 1} e_l G_|a|(r), so each charge row qhat^a is staged times
// c_a = (-1)^|a| (1, 1, 1, 3, 1, 3, 3, 15)_a and the radial factors lose those constants:
// Coulomb G_0 = 1/r, G_1 = 1/r^3, G_2 / 3 = 1/r^5, G_3 / 15 = 1/r^7; Yukawa multiplies them by
// e^{-kr} (1, 1 + kr, 1 + kr + (kr)^2/3, 1 + kr + (2/5)(kr)^2 + (kr)^3/15).  The tensor grid
// is walked as in far_mixed (e_x^2 + e_y^2 and e_x e_y per (k1, k2) row); runs of rows are
// summed in FP32 and folded into the caller's TwoSum accumulator.
template <int KER>
__device__ void far_hermite_mixed(const SweepArgs& a, int C, const double cb[3], const Targets& tg,
                                  float (&hi)[kT], float (&lo)[kT], float2* sm, int g, int G) {
    const int np1 = a.np1, n = np1 - 1, P = np1 * np1 * np1;
    const float* qh = a.qhat32 + static_cast<int64_t>(a.qslot[C]) * 8 * P;
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * np1; k += kThreads) {
        const int d = k / np1, kk = k - d * np1;
        const double s = cheb_point(a.cheb_t, kk, n, a.s_lo[3 * C + d], a.s_hi[3 * C + d]);
        const float v = __double2float_rn(s - (d == 0 ? cb[0] : (d == 1 ? cb[1] : cb[2])));
        sm[k] = make_float2(v, v);
    }
    float2* sq = sm + 3 * np1;
    for (int k = threadIdx.x; k < 8 * P; k += kThreads) {
        const int c = k / P;
        const float w = (c == 0) ? 1.f : (c == 7) ? -15.f : (c == 3 || c == 5 || c == 6) ? 3.f : -1.f;
        const float v = w * qh[k];
        sq[k] = make_float2(v, v);
    }
    __syncthreads();
    const float2* sxp = sm;
    const float2* syp = sm + np1;
    const float2* szp = sm + 2 * np1;
    const float2 nk = make_float2(a.neg_kappa_log2e, a.neg_kappa_log2e);
    const float2 kp = make_float2(a.param32, a.param32);
    const int R = np1 * np1, run = max(1, kBlock / (8 * np1)) * G;
    int k1 = g / np1, k2 = g - k1 * np1;
    for (int row0 = g; row0 < R; row0 += run) {
        float2 f[kH];
#pragma unroll
        for (int v = 0; v < kH; ++v) f[v] = make_float2(0.f, 0.f);
        for (int row = row0; row < min(R, row0 + run); row += G) {
            const float2 sx = sxp[k1], sy = syp[k2];
            float2 ex[kH], ey[kH], t[kH];
#pragma unroll
            for (int v = 0; v < kH; ++v) {
                ex[v] = add2(sx, tg.x[v]);
                ey[v] = add2(sy, tg.y[v]);
                t[v] = fma2(ey[v], ey[v], mul2(ex[v], ex[v]));
            }
            const float2* qrow = sq + row * np1;
            for (int k3 = 0; k3 < np1; ++k3) {
                const float2 sz = szp[k3];
                float2 q[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) q[c] = qrow[c * P + k3];
#pragma unroll
                for (int v = 0; v < kH; ++v) {
                    const float2 ez = add2(sz, tg.z[v]);
                    const float2 r2 = fma2(ez, ez, t[v]);
                    float2 g0 = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
                    const float2 ri2 = mul2(g0, g0);
                    float2 g1 = mul2(g0, ri2), g2 = mul2(g1, ri2), g3 = mul2(g2, ri2);
                    if (KER == BLTC_KERNEL_YUKAWA) {
                        const float2 r = mul2(r2, g0);
                        const float2 x = mul2(nk, r);
                        const float2 e = make_float2(ex2_approx(x.x), ex2_approx(x.y));
                        const float2 kr = mul2(kp, r);
                        const float2 one = make_float2(1.f, 1.f);
                        const float2 p1 = add2(one, kr);
                        const float2 p2 = fma2(mul2(kr, kr), make_float2(1.f / 3.f, 1.f / 3.f), p1);
                        const float2 p3 = fma2(mul2(kr, kr), fma2(kr, make_float2(1.f / 15.f, 1.f / 15.f),
                                                                  make_float2(0.4f, 0.4f)), p1);
                        g0 = mul2(g0, e);
                        g1 = mul2(mul2(g1, e), p1);
                        g2 = mul2(mul2(g2, e), p2);
                        g3 = mul2(mul2(g3, e), p3);
                    }
                    const float2 s1 = fma2(ez, q[1], fma2(ey[v], q[2], mul2(ex[v], q[4])));
                    const float2 exy = mul2(ex[v], ey[v]);
                    const float2 s2 = fma2(ez, fma2(ey[v], q[3], mul2(ex[v], q[5])), mul2(exy, q[6]));
                    const float2 s3 = mul2(mul2(exy, ez), q[7]);
                    f[v] = fma2(g0, q[0], f[v]);
                    f[v] = fma2(g1, s1, f[v]);
                    f[v] = fma2(g2, s2, f[v]);
                    f[v] = fma2(g3, s3, f[v]);
                }
            }
            for (k2 += G; k2 >= np1; k2 -= np1) ++k1;
        }
#pragma unroll
        for (int v = 0; v < kH; ++v) {
            two_sum_add(hi[2 * v], lo[2 * v], f[v].x);
            two_sum_add(hi[2 * v + 1], lo[2 * v + 1], f[v].y);
        }
    }
}

template <int KER, bool HERM = false>
__device__ void item_mixed(const SweepArgs& a, int4 it, float4* sm) {
    const int b = it.x;
    const int B = a.b_leaves[b];
    const int tb = a.b_begin[B], nb = a.b_count[B];
    const double cb[3] = {a.b_center[3 * B], a.b_center[3 * B + 1], a.b_center[3 * B + 2]};
    const int a0 = a.app_off[b], na = a.app_off[b + 1] - a0, d0 = a.dir_off[b];
    double* out = a.partials + a.part_off[b] + static_cast<int64_t>(it.w) * nb;
    const int G = groups_for(nb, a.g_max);
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
        {   // far field: an item lists its approximated clusters (e < na) before its leaves
            float fh[kT], fl[kT];
#pragma unroll
            for (int u = 0; u < kT; ++u) fh[u] = fl[u] = 0.f;
            for (int e = it.y; e < min(it.z, na); ++e) {
                if constexpr (HERM)
                    far_hermite_mixed<KER>(a, a.app_ids[a0 + e], cb, tg, fh, fl, reinterpret_cast<float2*>(sm), g, G);
                else
                    far_mixed<KER>(a, a.app_ids[a0 + e], cb, tg, fh, fl, reinterpret_cast<float2*>(sm), g, G);
            }
#pragma unroll
            for (int u = 0; u < kT; ++u) acc[u * kThreads] += static_cast<double>(fh[u]) + static_cast<double>(fl[u]);
        }
        for (int e = max(it.y, na); e < it.z; ++e) {
            const int de = d0 + e - na;
            const int C = a.dir_ids[de];
            const float tau2 = a.dir_tau2[de];
            const uint8_t sel = a.dir_sel[de];
            if (sel & kSelSkip) continue;            // evaluated by the partner's mutual entry
            if (sel & kSelMutual) {
                float* sbuf = reinterpret_cast<float*>(reinterpret_cast<char*>(sm) + kSmemBytes + kAccBytes);
                float* mrow = a.mpart + a.dir_moff[de];
                switch (sel & (kSelZero | kSelClose)) {
                    case 0: near_mutual<KER, false, false>(a, C, B, tau2, cb, tg, acc, sm, sbuf, mrow, g, G, tb, nb, t0, l, tpg); break;
                    case kSelClose: near_mutual<KER, false, true>(a, C, B, tau2, cb, tg, acc, sm, sbuf, mrow, g, G, tb, nb, t0, l, tpg); break;
                    default: near_mutual<KER, true, true>(a, C, B, tau2, cb, tg, acc, sm, sbuf, mrow, g, G, tb, nb, t0, l, tpg); break;
                }
                continue;
            }
            switch (sel & (kSelZero | kSelClose)) {
                case 0: near_mixed<KER, false, false>(a, C, B, tau2, cb, tg, acc, sm, g, G, tb, nb, t0, l, tpg); break;
                case kSelClose: near_mixed<KER, false, true>(a, C, B, tau2, cb, tg, acc, sm, g, G, tb, nb, t0, l, tpg); break;
                default: near_mixed<KER, true, true>(a, C, B, tau2, cb, tg, acc, sm, g, G, tb, nb, t0, l, tpg); break;
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


// The persistent mixed sweep: blocks pull (batch, list range) items from an atomic counter.
template <int KER, bool HERM = false>
__device__ __forceinline__ void sweep_mixed_body(const SweepArgs& a) {
    extern __shared__ __align__(16) float4 sm_dyn[];
    float4* sm = sm_dyn;
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = static_cast<int>(atomicAdd(a.counter, 1u));
        __syncthreads();
        const int i = s_item;
        if (i >= a.n_items) return;
        item_mixed<KER, HERM>(a, a.items[i], sm);
    }
}

// ---- FP64 ---------------------------------------------------------------------------

template <int KER>
__device__ __forceinline__ double g_fp64(double r2, double q, double kappa) {
    return q * g64<KER>(r2, kappa);
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
__device__ __forceinline__ void sweep_fp64_body(const SweepArgs& a) {
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

// ---- barycentric Hermite far field (FP64) ------------------------------------------------

// The radial factors G_m(r), m = 0..3, of the mixed derivatives D^a G = prod_{a_l} d_l G_|a|
// (d = x - y; G_{m+1} = -G_m'/r): Coulomb 1/r, 1/r^3, 3/r^5, 15/r^7 and Yukawa
// e^{-kr}(1, 1 + kr, 3 + 3kr + (kr)^2, 15 + 15kr + 6(kr)^2 + (kr)^3) / r^(2m+1).
template <int KER>
__device__ __forceinline__ void hermite_radial(double r2, double kappa, double (&g)[4]) {
    const double ri = rsqrt(r2);
    const double ri2 = ri * ri;
    double e = 1.0, kr = 0.0;
    if (KER == BLTC_KERNEL_YUKAWA) {
        kr = kappa * (r2 * ri);
        e = exp(-kr);
    }
    g[0] = e * ri;
    g[1] = g[0] * ri2 * (1.0 + kr);
    g[2] = e * ri * ri2 * ri2 * (3.0 + 3.0 * kr + kr * kr);
    g[3] = e * ri * ri2 * ri2 * ri2 * (15.0 + 15.0 * kr + 6.0 * kr * kr + kr * kr * kr);
}

// Far field of cluster C with Hermite modified charges qhat^a_k (a = a1*4 + a2*2 + a3, 8 rows
// of (n+1)^3 in a.qhat64 at slot a.qslot[C]): phi_i += sum_k sum_a D^a G(x_i, s_k) qhat^a_k.
template <int KER, int T>
__device__ void far_hermite_fp64(const SweepArgs& a, int C, const double (&xt)[T], const double (&yt)[T],
                                 const double (&zt)[T], double (&acc)[T], double* sm) {
    const int np1 = a.np1, n = np1 - 1, P = np1 * np1 * np1;
    const double* qh = a.qhat64 + static_cast<int64_t>(a.qslot[C]) * 8 * P;
    __syncthreads();
    for (int k = threadIdx.x; k < 3 * np1; k += kThreads) {
        const int d = k / np1, kk = k - d * np1;
        sm[k] = cheb_point(a.cheb_t, kk, n, a.s_lo[3 * C + d], a.s_hi[3 * C + d]);
    }
    double* sq = sm + 3 * np1;
    for (int k = threadIdx.x; k < 8 * P; k += kThreads) sq[k] = qh[k];
    __syncthreads();
    for (int k1 = 0; k1 < np1; ++k1) {
        for (int k2 = 0; k2 < np1; ++k2) {
            for (int k3 = 0; k3 < np1; ++k3) {
                const int k = (k1 * np1 + k2) * np1 + k3;
                double qa[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) qa[c] = sq[c * P + k];
#pragma unroll
                for (int u = 0; u < T; ++u) {
                    const double d0 = xt[u] - sm[k1], d1 = yt[u] - sm[np1 + k2], d2 = zt[u] - sm[2 * np1 + k3];
                    const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                    if (r2 == 0.0) continue;                    // as the direct sum (skipped pair)
                    double g[4];
                    hermite_radial<KER>(r2, a.kappa, g);
                    const double d01 = d0 * d1, d02 = d0 * d2, d12 = d1 * d2;
                    acc[u] += g[0] * qa[0] + g[1] * (d2 * qa[1] + d1 * qa[2] + d0 * qa[4]) +
                              g[2] * (d12 * qa[3] + d02 * qa[5] + d01 * qa[6]) + g[3] * (d01 * d2) * qa[7];
                }
            }
        }
    }
}

template <int KER, int T>
__device__ void item_hermite(const SweepArgs& a, int4 it, D4* sm) {
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
                far_hermite_fp64<KER, T>(a, a.app_ids[a0 + e], xt, yt, zt, acc, reinterpret_cast<double*>(sm));
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
__device__ __forceinline__ void sweep_hermite_body(const SweepArgs& a) {
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
            item_hermite<KER, 1>(a, it, sm);
        else
            item_hermite<KER, 2>(a, it, sm);
    }
}

}  // namespace sweepdev
}  // namespace bltc
