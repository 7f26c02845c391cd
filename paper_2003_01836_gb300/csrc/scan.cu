// scan.cu -- device-wide exclusive prefix sums used to turn per-item counts into offsets
// (tree chunks, list CSR offsets, work-item and partial-sum layouts).
#include "internal.cuh"

namespace bltc {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 4;
constexpr int kTile = kThreads * kPerThread;

template <typename T>
__device__ T block_exclusive_scan(T v, T* warp_sums, T* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (blockDim.x >> 5) ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (blockDim.x >> 5)) warp_sums[lane] = w;  // inclusive over warps
    }
    __syncthreads();
    T before = warp == 0 ? T(0) : warp_sums[warp - 1];
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    T r = before + x - v;
    __syncthreads();
    return r;
}

template <typename T>
__global__ void k_scan_tiles(const T* __restrict__ in, T* __restrict__ out,
                             T* __restrict__ sums, int64_t n) {
    __shared__ T ws[32];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile + threadIdx.x * kPerThread;
    T v[kPerThread];
    T local = 0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        v[k] = (base + k < n) ? in[base + k] : T(0);
        local += v[k];
    }
    T tot;
    T run = block_exclusive_scan<T>(local, ws, &tot);
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// One block scans the per-tile sums in place (sequential carry across 1024-wide slabs).
template <typename T>
__global__ void k_scan_sums(T* __restrict__ sums, int64_t m, T* __restrict__ total) {
    __shared__ T ws[32];
    __shared__ T carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t s = 0; s < m; s += blockDim.x) {
        int64_t i = s + threadIdx.x;
        T v = i < m ? sums[i] : T(0);
        T tot;
        T ex = block_exclusive_scan<T>(v, ws, &tot);
        if (i < m) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void k_scan_add(T* __restrict__ out, const T* __restrict__ sums, int64_t n) {
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kTile;
    const T add = sums[blockIdx.x];
    for (int k = threadIdx.x; k < kTile; k += kThreads)
        if (base + k < n) out[base + k] += add;
}

template <typename T>
void scan_impl(Context* ctx, const T* in, T* out, int64_t n, T* total) {
    if (n <= 0) {
        if (total) BLTC_CUDA(cudaMemsetAsync(total, 0, sizeof(T), ctx->stream));
        return;
    }
    const int64_t tiles = ceil_div(n, kTile);
    DBuf<T> sums(ctx, tiles);
    k_scan_tiles<T><<<static_cast<unsigned>(tiles), kThreads, 0, ctx->stream>>>(in, out, sums.p, n); ++ctx->launches;
    BLTC_LAUNCH_CHECK("scan_tiles");
    k_scan_sums<T><<<1, 1024, 0, ctx->stream>>>(sums.p, tiles, total); ++ctx->launches;
    BLTC_LAUNCH_CHECK("scan_sums");
    if (tiles > 1) {
        k_scan_add<T><<<static_cast<unsigned>(tiles), kThreads, 0, ctx->stream>>>(out, sums.p, n); ++ctx->launches;
        BLTC_LAUNCH_CHECK("scan_add");
    }
}

}  // namespace

void exclusive_scan_i32(Context* ctx, const int32_t* in, int32_t* out, int64_t n,
                        int32_t* total) {
    scan_impl<int32_t>(ctx, in, out, n, total);
}

void exclusive_scan_i64(Context* ctx, const int64_t* in, int64_t* out, int64_t n,
                        int64_t* total) {
    scan_impl<int64_t>(ctx, in, out, n, total);
}

}  // namespace bltc
