// direct.cu -- O(N^2) direct summation of Eq. 1 on the GPU (the baseline the treecode is
// compared with; the paper computed it as one batch-cluster direct-sum launch over all
// targets and all sources, Sec. IV "Single GPU vs. Single 6-Core CPU").
//
// Grid: (target tiles of 256*T targets) x (source splits).  Each block stages its sources
// in shared-memory tiles and streams them against the targets held in registers, writing
// one partial per (split, target) into a scratch buffer; a second kernel sums the splits
// in order, so the result does not depend on scheduling.  MIXED evaluates in FP32 with every
// coordinate an FP32 (hi, lo) pair, sums blocks of sources in FP32 and tiles in FP64.
#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace bltc {
namespace {

constexpr int kThreads = 256;
constexpr int kTileM = 512;      // sources per staged tile of the MIXED kernel (64 B each)
constexpr int kTile64 = 1024;
constexpr int kBlock = 32;       // FP32 block folded into a TwoSum accumulator

struct DirectArgs {
    const double *tx, *ty, *tz;
    const double *sx, *sy, *sz, *sq;
    int64_t nt, ns, per_split;
    double* partial;            // [splits * nt]
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

// Knuth's TwoSum fold of a short FP32 block sum into a compensated FP32 accumulator.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

// An FP64 value as an FP32 pair hi + lo (hi = fp32(v), lo = fp32(v - hi)): about 48 bits.
__device__ __forceinline__ float2 split_pair(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - static_cast<double>(h)));
}

// MIXED: every coordinate enters as an FP32 pair, and x_j - x_i = (hi_j - hi_i) + (lo_j - lo_i).
// For a close pair the two highs are within a factor of two of each other, so their
// difference is exact (Sterbenz) and the distance keeps FP32's relative precision however
// close the particles are; with coordinates rounded once to FP32, a pair at distance r would
// carry a relative error of about 2^-24 |x| / r.  Two targets per packed FP32x2 operation;
// the FP32 sums over blocks of kBlock sources are folded by TwoSum, tiles are added in FP64.
template <int KER, int T>
__global__ void __launch_bounds__(kThreads, 2) k_direct_mixed(DirectArgs a) {
    static_assert(T % 2 == 0, "targets are processed in packed pairs");
    constexpr int H = T / 2;
    // per source: (xh, xh, yh, yh), (zh, zh, q, q), (xl, xl, yl, yl), (zl, zl, 0, 0)
    __shared__ __align__(16) float4 sm[4 * kTileM];
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * kThreads * T;
    const int64_t s0 = static_cast<int64_t>(blockIdx.y) * a.per_split;
    const int64_t s1 = std::min<int64_t>(a.ns, s0 + a.per_split);
    float2 nxh[H], nyh[H], nzh[H], nxl[H], nyl[H], nzl[H];   // targets, negated
    double acc[T];
#pragma unroll
    for (int u = 0; u < T; ++u) {
        const int64_t t = std::min<int64_t>(t0 + threadIdx.x + kThreads * u, a.nt - 1);
        const float2 px = split_pair(a.tx[t]), py = split_pair(a.ty[t]), pz = split_pair(a.tz[t]);
        if (u & 1) {
            nxh[u / 2].y = -px.x; nxl[u / 2].y = -px.y;
            nyh[u / 2].y = -py.x; nyl[u / 2].y = -py.y;
            nzh[u / 2].y = -pz.x; nzl[u / 2].y = -pz.y;
        } else {
            nxh[u / 2].x = -px.x; nxl[u / 2].x = -px.y;
            nyh[u / 2].x = -py.x; nyl[u / 2].x = -py.y;
            nzh[u / 2].x = -pz.x; nzl[u / 2].x = -pz.y;
        }
        acc[u] = 0.0;
    }
    const float2 nkl2e = make_float2(a.neg_kappa_log2e, a.neg_kappa_log2e);
    for (int64_t j0 = s0; j0 < s1; j0 += kTileM) {
        const int m = static_cast<int>(std::min<int64_t>(kTileM, s1 - j0));
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += kThreads) {
            const float2 px = split_pair(a.sx[j0 + j]), py = split_pair(a.sy[j0 + j]);
            const float2 pz = split_pair(a.sz[j0 + j]);
            const float q = __double2float_rn(a.sq[j0 + j]);
            sm[4 * j] = make_float4(px.x, px.x, py.x, py.x);
            sm[4 * j + 1] = make_float4(pz.x, pz.x, q, q);
            sm[4 * j + 2] = make_float4(px.y, px.y, py.y, py.y);
            sm[4 * j + 3] = make_float4(pz.y, pz.y, 0.f, 0.f);
        }
        __syncthreads();
        float hi[T], lo[T];
#pragma unroll
        for (int u = 0; u < T; ++u) hi[u] = lo[u] = 0.f;
        for (int jb = 0; jb < m; jb += kBlock) {
            const int je = min(jb + kBlock, m);
            float2 f[H];
#pragma unroll
            for (int v = 0; v < H; ++v) f[v] = make_float2(0.f, 0.f);
#pragma unroll 2
            for (int j = jb; j < je; ++j) {
                const float4 h0 = sm[4 * j], h1 = sm[4 * j + 1], l0 = sm[4 * j + 2], l1 = sm[4 * j + 3];
                const float2 sxh = make_float2(h0.x, h0.y), syh = make_float2(h0.z, h0.w);
                const float2 szh = make_float2(h1.x, h1.y), sq = make_float2(h1.z, h1.w);
                const float2 sxl = make_float2(l0.x, l0.y), syl = make_float2(l0.z, l0.w);
                const float2 szl = make_float2(l1.x, l1.y);
#pragma unroll
                for (int v = 0; v < H; ++v) {
                    const float2 dx = __fadd2_rn(__fadd2_rn(sxh, nxh[v]), __fadd2_rn(sxl, nxl[v]));
                    const float2 dy = __fadd2_rn(__fadd2_rn(syh, nyh[v]), __fadd2_rn(syl, nyl[v]));
                    const float2 dz = __fadd2_rn(__fadd2_rn(szh, nzh[v]), __fadd2_rn(szl, nzl[v]));
                    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                    float2 ri = make_float2(r2.x > 0.f ? rsqrt_approx(r2.x) : 0.f,
                                            r2.y > 0.f ? rsqrt_approx(r2.y) : 0.f);
                    if (KER == BLTC_KERNEL_YUKAWA) {
                        const float2 e = __fmul2_rn(nkl2e, __fmul2_rn(r2, ri));
                        ri = __fmul2_rn(ri, make_float2(ex2_approx(e.x), ex2_approx(e.y)));
                    }
                    f[v] = __ffma2_rn(sq, ri, f[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < H; ++v) {
                two_sum_add(hi[2 * v], lo[2 * v], f[v].x);
                two_sum_add(hi[2 * v + 1], lo[2 * v + 1], f[v].y);
            }
        }
#pragma unroll
        for (int u = 0; u < T; ++u) acc[u] += static_cast<double>(hi[u]) + static_cast<double>(lo[u]);
    }
    double* out = a.partial + static_cast<int64_t>(blockIdx.y) * a.nt;
#pragma unroll
    for (int u = 0; u < T; ++u) {
        const int64_t t = t0 + threadIdx.x + kThreads * u;
        if (t < a.nt) out[t] = acc[u];
    }
}

template <int KER, int T>
__global__ void __launch_bounds__(kThreads, 2) k_direct_fp64(DirectArgs a) {
    __shared__ __align__(16) D4 sm[kTile64];
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * kThreads * T;
    const int64_t s0 = static_cast<int64_t>(blockIdx.y) * a.per_split;
    const int64_t s1 = std::min<int64_t>(a.ns, s0 + a.per_split);
    double xt[T], yt[T], zt[T], acc[T];
#pragma unroll
    for (int u = 0; u < T; ++u) {
        const int64_t t = std::min<int64_t>(t0 + threadIdx.x + kThreads * u, a.nt - 1);
        xt[u] = a.tx[t];
        yt[u] = a.ty[t];
        zt[u] = a.tz[t];
        acc[u] = 0.0;
    }
    for (int64_t j0 = s0; j0 < s1; j0 += kTile64) {
        const int m = static_cast<int>(std::min<int64_t>(kTile64, s1 - j0));
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += kThreads)
            sm[j] = D4{a.sx[j0 + j], a.sy[j0 + j], a.sz[j0 + j], a.sq[j0 + j]};
        __syncthreads();
        for (int j = 0; j < m; ++j) {
            const D4 s = sm[j];
#pragma unroll
            for (int u = 0; u < T; ++u) {
                const double dx = xt[u] - s.x, dy = yt[u] - s.y, dz = zt[u] - s.z;
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 != 0.0) {
                    double ri = rsqrt(r2);
                    if (KER == BLTC_KERNEL_YUKAWA) ri *= exp(-a.kappa * (r2 * ri));
                    acc[u] += s.w * ri;
                }
            }
        }
    }
    double* out = a.partial + static_cast<int64_t>(blockIdx.y) * a.nt;
#pragma unroll
    for (int u = 0; u < T; ++u) {
        const int64_t t = t0 + threadIdx.x + kThreads * u;
        if (t < a.nt) out[t] = acc[u];
    }
}

__global__ void k_direct_reduce(const double* __restrict__ partial, int64_t nt, int splits,
                                double* __restrict__ phi) {
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < nt;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < splits; ++k) s += partial[static_cast<int64_t>(k) * nt + t];
        phi[t] = s;
    }
}

// Scratch of bltc_direct_sum_noalloc: the per-split partial sums live in this fixed
// file-scope array instead of memory from an allocator.  Every GPU that loads the library
// holds it (64 MiB) until the process exits.
constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 23;
__device__ __align__(256) double g_direct_scratch[kNoAllocScratchDoubles];

// Device address of g_direct_scratch on `device`, looked up once per device with that device
// current (host code must not use the symbol itself as a device pointer).
double* direct_scratch_address(int device) {
    static std::mutex mu;
    static double* addr[256] = {};
    if (device < 0 || device >= 256) throw Error(BLTC_ERR_ARG, "direct noalloc: device out of range");
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_direct_scratch);
        if (e != cudaSuccess)
            throw Error(BLTC_ERR_CUDA, std::string("cudaGetSymbolAddress(g_direct_scratch): ") +
                                           cudaGetErrorString(e));
        addr[device] = static_cast<double*>(p);
    }
    return addr[device];
}

}  // namespace

void direct_sum(Context* ctx, const double* tx, const double* ty, const double* tz, int64_t nt,
                const double* sx, const double* sy, const double* sz, const double* sq,
                int64_t ns, const bltc_params& p, double* phi) {
    require(nt >= 1 && ns >= 1, "direct: nt and ns must be >= 1");
    require(tx && ty && tz && sx && sy && sz && sq && phi, "direct: NULL pointer");
    cudaStream_t s = ctx->stream;
    const bool mixed = p.precision == BLTC_PRECISION_MIXED;
    const int T = 4;
    const int64_t tiles = ceil_div(nt, static_cast<int64_t>(kThreads) * T);
    const int64_t want = 4 * static_cast<int64_t>(std::max(1, ctx->sm_count));
    const int64_t tile_src = mixed ? kTileM : kTile64;
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>(ceil_div(want, tiles), ceil_div(ns, tile_src)));
    splits = std::min<int64_t>(splits, 65535);
    const int64_t per = ceil_div(ceil_div(ns, splits), tile_src) * tile_src;
    splits = ceil_div(ns, per);
    DBuf<double> partial(ctx, splits * nt);
    DirectArgs a{tx, ty, tz, sx, sy, sz, sq, nt, ns, per, partial.p, 0.0, 0.f};
    const double kappa = p.kernel == BLTC_KERNEL_YUKAWA ? p.kappa : 0.0;
    a.kappa = kappa;
    a.neg_kappa_log2e = static_cast<float>(-kappa * 1.4426950408889634);
    const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(splits));
    if (mixed) {
        if (p.kernel == BLTC_KERNEL_YUKAWA) {
            k_direct_mixed<BLTC_KERNEL_YUKAWA, 4><<<grid, kThreads, 0, s>>>(a); ++ctx->launches;
        }
        else {
            k_direct_mixed<BLTC_KERNEL_COULOMB, 4><<<grid, kThreads, 0, s>>>(a); ++ctx->launches;
        }
    } else {
        if (p.kernel == BLTC_KERNEL_YUKAWA) {
            k_direct_fp64<BLTC_KERNEL_YUKAWA, 4><<<grid, kThreads, 0, s>>>(a); ++ctx->launches;
        }
        else {
            k_direct_fp64<BLTC_KERNEL_COULOMB, 4><<<grid, kThreads, 0, s>>>(a); ++ctx->launches;
        }
    }
    BLTC_LAUNCH_CHECK("direct");
    k_direct_reduce<<<grid_for(nt, 256, 4096), 256, 0, s>>>(partial.p, nt, static_cast<int>(splits), phi); ++ctx->launches;
    BLTC_LAUNCH_CHECK("direct reduce");
}

void direct_sum_noalloc(Context* ctx, const double* tx, const double* ty, const double* tz,
                        int64_t nt, const double* sx, const double* sy, const double* sz,
                        const double* sq, int64_t ns, const bltc_params& p, double* phi) {
    require(nt >= 1 && ns >= 1, "direct noalloc: nt and ns must be >= 1");
    require(tx && ty && tz && sx && sy && sz && sq && phi, "direct noalloc: NULL pointer");
    require(nt <= kNoAllocScratchDoubles,
            "direct noalloc: nt exceeds the scratch capacity of 8388608 targets");
    double* scratch = direct_scratch_address(ctx->device);
    cudaStream_t s = ctx->stream;
    const bool mixed = p.precision == BLTC_PRECISION_MIXED;
    const int T = 4;
    const int64_t tiles = ceil_div(nt, static_cast<int64_t>(kThreads) * T);
    const int64_t want = 4 * static_cast<int64_t>(std::max(1, ctx->sm_count));
    const int64_t tile_src = mixed ? kTileM : kTile64;
    // as many source splits as the fixed scratch holds (splits * nt partial sums)
    int64_t splits = std::max<int64_t>(1, std::min<int64_t>(ceil_div(want, tiles), ceil_div(ns, tile_src)));
    splits = std::min<int64_t>({splits, int64_t(65535), kNoAllocScratchDoubles / nt});
    const int64_t per = ceil_div(ceil_div(ns, splits), tile_src) * tile_src;
    splits = ceil_div(ns, per);
    DirectArgs a{tx, ty, tz, sx, sy, sz, sq, nt, ns, per, scratch, 0.0, 0.f};
    const double kappa = p.kernel == BLTC_KERNEL_YUKAWA ? p.kappa : 0.0;
    a.kappa = kappa;
    a.neg_kappa_log2e = static_cast<float>(-kappa * 1.4426950408889634);
    const dim3 grid(static_cast<unsigned>(tiles), static_cast<unsigned>(splits));
    if (mixed) {
        if (p.kernel == BLTC_KERNEL_YUKAWA)
            k_direct_mixed<BLTC_KERNEL_YUKAWA, 4><<<grid, kThreads, 0, s>>>(a);
        else
            k_direct_mixed<BLTC_KERNEL_COULOMB, 4><<<grid, kThreads, 0, s>>>(a);
    } else {
        if (p.kernel == BLTC_KERNEL_YUKAWA)
            k_direct_fp64<BLTC_KERNEL_YUKAWA, 4><<<grid, kThreads, 0, s>>>(a);
        else
            k_direct_fp64<BLTC_KERNEL_COULOMB, 4><<<grid, kThreads, 0, s>>>(a);
    }
    ++ctx->launches;
    BLTC_LAUNCH_CHECK("direct noalloc");
    k_direct_reduce<<<grid_for(nt, 256, 4096), 256, 0, s>>>(scratch, nt, static_cast<int>(splits), phi);
    ++ctx->launches;
    BLTC_LAUNCH_CHECK("direct noalloc reduce");
}

}  // namespace bltc
