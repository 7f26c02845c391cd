// tree.cu -- A0: the tree of source clusters / target batches on the GPU.
//
// Sec. II-D: the root is the minimal bounding box of the particles; every cluster holding
// more than max_leaf particles is divided at the midpoint of its box.  Sec. III-A: a
// cluster is cut into 8 children, or into 2 or 4 when more would leave an aspect ratio
// above sqrt(2).  The exact rules (which dimensions split, ties, child order, stable
// particle order, DFS pre-order ids, when a node stays a leaf) are stated in bltc.h.
//
// The build is level-synchronous.  For each level: (1) every node decodes its box, centre,
// radius and split; (2) its particles, cut into fixed-size chunks, are classified into
// octants with a per-chunk histogram; (3) one block per node scans its chunk histograms,
// decides leaf or split, and creates the children with their particle ranges; (4) every
// chunk scatters its particles stably into the children's ranges (or copies a finished
// leaf's particles to the output) while reducing the children's boxes with atomics.  The
// host reads two counters per level.  Afterwards subtree sizes give DFS pre-order ids.
//
// Everything that decides the tree is exact FP64 (compare, min/max, and the IEEE-rounded
// +, -, *, sqrt intrinsics); this file is also compiled with --fmad=false.
#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace bltc {
namespace {

constexpr int kCh = 2048;        // particles per chunk
constexpr int kThreads = 256;

struct BNode {                   // a node in creation (BFS) order
    unsigned long long key[6];   // ordered keys of min x,y,z and max x,y,z
    double lo[3], hi[3], center[3], mid[3];
    double radius;
    int32_t begin, count, parent, level;
    int32_t nch, split, chunk0, nchunk;
    int32_t child[8];            // BFS ids in increasing octant order
    int32_t octbase[8];          // first tree position of each octant's particles
    int32_t octchild[8];         // octant -> BFS id of its child (or -1)
    int32_t dfs, size;
};

struct BChunk {
    int32_t node, start, end, pad;
    int32_t hist[8];
    int32_t prefix[8];           // particles of each octant in the node's earlier chunks
};

// Order-preserving map of a double to an unsigned key; -0.0 sorts just below +0.0.
__device__ __forceinline__ unsigned long long okey(double v) {
    unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}
__device__ __forceinline__ double okey_inv(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffULL) : ~k;
    return __longlong_as_double(static_cast<long long>(b));
}

__device__ __forceinline__ void init_keys(BNode& nd) {
    for (int d = 0; d < 3; ++d) {
        nd.key[d] = ~0ULL;
        nd.key[3 + d] = 0ULL;
    }
}

__global__ void k_root_init(BNode* nodes, int32_t n, int32_t* counters) {
    counters[0] = 1;   // next node id
    counters[1] = 0;   // next chunk
    counters[2] = 0;   // bad-input flag
    counters[3] = 0;
    BNode& r = nodes[0];
    init_keys(r);
    r.begin = 0;
    r.count = n;
    r.parent = -1;
    r.level = 0;
    r.nch = 0;
    r.split = 0;
    r.chunk0 = 0;
    r.nchunk = static_cast<int32_t>((n + kCh - 1) / kCh);
    for (int c = 0; c < 8; ++c) r.child[c] = r.octchild[c] = -1;
}

__global__ void k_root_chunks(BChunk* chunks, int32_t n) {
    int64_t c = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t nc = (n + kCh - 1) / kCh;
    if (c >= nc) return;
    chunks[c].node = 0;
    chunks[c].start = static_cast<int32_t>(c * kCh);
    chunks[c].end = static_cast<int32_t>((c + 1) * kCh < n ? (c + 1) * kCh : n);
}

// Block-wide min and max of six keys, then one atomic per key into `dst`.
__device__ void block_box_atomic(unsigned long long mn[3], unsigned long long mx[3],
                                 unsigned long long* dst) {
    __shared__ unsigned long long s[6][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            mn[d] = min(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = max(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
        if (lane == 0) {
            s[d][warp] = mn[d];
            s[3 + d][warp] = mx[d];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        unsigned long long v = s[threadIdx.x][0];
        for (int w = 1; w < kThreads / 32; ++w)
            v = threadIdx.x < 3 ? min(v, s[threadIdx.x][w]) : max(v, s[threadIdx.x][w]);
        if (threadIdx.x < 3)
            atomicMin(&dst[threadIdx.x], v);
        else
            atomicMax(&dst[threadIdx.x], v);
    }
    __syncthreads();
}

// Copies the caller's particles into working buffer A (identity permutation), reduces the
// root box and flags non-finite input.
__global__ void k_root_copy(const double* __restrict__ x, const double* __restrict__ y,
                            const double* __restrict__ z, const double* __restrict__ q,
                            int32_t n, double* ax, double* ay, double* az, double* aq,
                            int32_t* ai, BNode* nodes, int* bad) {
    unsigned long long mn[3] = {~0ULL, ~0ULL, ~0ULL}, mx[3] = {0ULL, 0ULL, 0ULL};
    bool ok = true;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double v[3] = {x[i], y[i], z[i]};
        ax[i] = v[0];
        ay[i] = v[1];
        az[i] = v[2];
        ai[i] = static_cast<int32_t>(i);
        if (q) {
            double qq = q[i];
            aq[i] = qq;
            ok = ok && isfinite(qq);
        }
        for (int d = 0; d < 3; ++d) {
            ok = ok && isfinite(v[d]);
            unsigned long long k = okey(v[d]);
            mn[d] = min(mn[d], k);
            mx[d] = max(mx[d], k);
        }
    }
    if (!ok) atomicOr(bad, 1);
    block_box_atomic(mn, mx, nodes[0].key);
}

// (1) Box, centre, radius and split of every node of the level.  Sized on the device the
// level's range comes from `dlv` ({first node, end node, chunks}); a raised overflow flag
// (`stop`) stops every further split, and on the last level allowed (`last`) a node that would
// split stays a leaf and raises the flag, so the tree is always complete.
__global__ void k_node_prepare(BNode* nodes, int32_t l0, int32_t l1, int32_t max_leaf,
                               const int32_t* dlv, int32_t* stop, bool last) {
    if (dlv) {
        l0 = dlv[0];
        l1 = dlv[1];
    }
    const bool halt = stop != nullptr && *stop != 0;
    for (int64_t v = l0 + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < l1;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        BNode& nd = nodes[v];
        double L[3], h2 = 0.0, Lmax = 0.0;
        for (int d = 0; d < 3; ++d) {
            double lo = okey_inv(nd.key[d]), hi = okey_inv(nd.key[3 + d]);
            nd.lo[d] = lo;
            nd.hi[d] = hi;
            nd.center[d] = __dmul_rn(0.5, __dadd_rn(lo, hi));
            nd.mid[d] = nd.center[d];
            double h = __dmul_rn(0.5, __dsub_rn(hi, lo));
            h2 = (d == 0) ? __dmul_rn(h, h) : __dadd_rn(h2, __dmul_rn(h, h));
            L[d] = __dsub_rn(hi, lo);
            if (L[d] > Lmax) Lmax = L[d];
        }
        nd.radius = __dsqrt_rn(h2);
        nd.nch = 0;
        for (int c = 0; c < 8; ++c) nd.child[c] = nd.octchild[c] = -1;
        int split = 0;
        if (nd.count > max_leaf && Lmax > 0.0) {
            for (int d = 0; d < 3; ++d)
                if (__dmul_rn(L[d], 1.4142135623730951) >= Lmax) split |= (1 << d);
        }
        if (split && (halt || last)) {
            if (last) atomicOr(stop, 1);
            split = 0;
        }
        nd.split = split;
    }
}

// (2) Octant of every particle of a splitting node, and the chunk's histogram.  One block
// per chunk (chunks beyond the grid in turn); a chunk with node -1 was reserved and not used.
__global__ void k_classify(BChunk* chunks, const BNode* __restrict__ nodes,
                           const double* __restrict__ ax, const double* __restrict__ ay,
                           const double* __restrict__ az, uint8_t* __restrict__ oct,
                           int64_t nck, const int32_t* dlv) {
    __shared__ int hist[8];
    if (dlv) nck = dlv[2];
    for (int64_t c = blockIdx.x; c < nck; c += gridDim.x) {
        const BChunk ch = chunks[c];
        if (ch.node < 0) continue;
        const BNode& nd = nodes[ch.node];
        const int split = nd.split;
        if (split == 0) continue;
        __syncthreads();   // the previous chunk's histogram is stored
        if (threadIdx.x < 8) hist[threadIdx.x] = 0;
        __syncthreads();
        const double mx = nd.mid[0], my = nd.mid[1], mz = nd.mid[2];
        for (int32_t i = ch.start + threadIdx.x; i < ch.end; i += blockDim.x) {
            int o = 0;
            if ((split & 1) && !(ax[i] < mx)) o |= 1;
            if ((split & 2) && !(ay[i] < my)) o |= 2;
            if ((split & 4) && !(az[i] < mz)) o |= 4;
            oct[i] = static_cast<uint8_t>(o);
            atomicAdd(&hist[o], 1);
        }
        __syncthreads();
        if (threadIdx.x < 8) chunks[c].hist[threadIdx.x] = hist[threadIdx.x];
    }
}

// Takes `count` consecutive entries from the counter *ctr unless that would pass `cap`, and
// returns the first one, or -1 (nothing taken).  The compare-and-swap retries only while other
// blocks take entries; a bound on them makes the call fail rather than wait longer.
__device__ int64_t reserve(int32_t* ctr, int64_t count, int64_t cap) {
    int64_t old = *reinterpret_cast<volatile int32_t*>(ctr);
    for (int it = 0; it < (1 << 20); ++it) {
        if (old + count > cap) return -1;
        const int32_t prev = atomicCAS(ctr, static_cast<int32_t>(old), static_cast<int32_t>(old + count));
        if (prev == old) return old;
        old = prev;
    }
    return -1;
}

__device__ int block_exclusive_scan_int(int v, int* ws, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < kThreads / 32 ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kThreads / 32) ws[lane] = w;
    }
    __syncthreads();
    int r = (warp ? ws[warp - 1] : 0) + x - v;
    *total = ws[kThreads / 32 - 1];
    __syncthreads();
    return r;
}

// (3) One block per node: per-octant prefix over the node's chunks, leaf-or-split, and
// creation of the children.  The children's chunks are reserved first, then their node ids;
// a reservation that would pass a capacity is not made: the node stays a leaf, the overflow
// flag is raised, and chunks already reserved are marked unused (node -1).
__global__ void k_node_split(BNode* nodes, int32_t l0, int32_t l1, BChunk* chunks, BChunk* next_chunks,
                             int32_t* counters /* [0] next node, [1] next chunk */,
                             const int32_t* dlv, int64_t node_cap, int64_t chunk_cap, int32_t* flag) {
    __shared__ int ws[kThreads / 32];
    __shared__ int tot[8];
    __shared__ int base_id, base_chunk[8];
    __shared__ int64_t dead0, deadn;
    if (dlv) {
        l0 = dlv[0];
        l1 = dlv[1];
    }
    for (int64_t v = l0 + static_cast<int64_t>(blockIdx.x); v < l1; v += gridDim.x) {
        BNode& nd = nodes[v];
        const bool splits = nd.split != 0;
        __syncthreads();   // every thread has read the flag before thread 0 may change it
        if (!splits) continue;
        int carry[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int32_t c0 = 0; c0 < nd.nchunk; c0 += kThreads) {
            int32_t c = nd.chunk0 + c0 + threadIdx.x;
            bool in = (c0 + threadIdx.x) < nd.nchunk;
            for (int o = 0; o < 8; ++o) {
                int h = in ? chunks[c].hist[o] : 0;
                int t;
                int ex = block_exclusive_scan_int(h, ws, &t);
                if (in) chunks[c].prefix[o] = carry[o] + ex;
                carry[o] += t;
            }
        }
        if (threadIdx.x == 0) {
            int nonempty = 0;
            int64_t need = 0;
            for (int o = 0; o < 8; ++o) {
                tot[o] = carry[o];
                nonempty += carry[o] > 0;
                need += (carry[o] + kCh - 1) / kCh;
            }
            base_id = -1;
            dead0 = deadn = 0;
            if (nonempty <= 1) {
                nd.split = 0;     // the split separates nothing: the node stays a leaf
            } else {
                const int64_t ck = reserve(&counters[1], need, chunk_cap);
                const int64_t id0 = ck >= 0 ? reserve(&counters[0], nonempty, node_cap) : -1;
                if (id0 < 0) {
                    atomicOr(flag, 1);
                    nd.split = 0;
                    if (ck >= 0) {
                        dead0 = ck;
                        deadn = need;
                    }
                } else {
                    nd.nch = nonempty;
                    base_id = static_cast<int>(id0);
                    int pos = nd.begin, c = 0;
                    int64_t chunk = ck;
                    for (int o = 0; o < 8; ++o) {
                        nd.octbase[o] = pos;
                        if (tot[o] > 0) {
                            int id = base_id + c;
                            nd.child[c] = id;
                            nd.octchild[o] = id;
                            BNode& k = nodes[id];
                            init_keys(k);
                            k.begin = pos;
                            k.count = tot[o];
                            k.parent = static_cast<int32_t>(v);
                            k.level = nd.level + 1;
                            k.nch = 0;
                            k.split = 0;
                            k.nchunk = (tot[o] + kCh - 1) / kCh;
                            k.chunk0 = static_cast<int32_t>(chunk);
                            chunk += k.nchunk;
                            base_chunk[o] = k.chunk0;
                            for (int j = 0; j < 8; ++j) k.child[j] = k.octchild[j] = -1;
                            ++c;
                        } else {
                            base_chunk[o] = -1;
                        }
                        pos += tot[o];
                    }
                }
            }
        }
        __syncthreads();
        for (int64_t j = threadIdx.x; j < deadn; j += blockDim.x) next_chunks[dead0 + j].node = -1;
        if (base_id >= 0) {
            for (int o = 0; o < 8; ++o) {
                if (tot[o] == 0) continue;
                const int id = nd.octchild[o], b = nd.octbase[o], nck = (tot[o] + kCh - 1) / kCh;
                for (int j = threadIdx.x; j < nck; j += blockDim.x) {
                    BChunk& ch = next_chunks[base_chunk[o] + j];
                    ch.node = id;
                    ch.start = b + j * kCh;
                    ch.end = min(b + tot[o], b + (j + 1) * kCh);
                }
            }
        }
        __syncthreads();   // the shared state is reused by the next node
    }
}

// (4) Stable scatter of each chunk into its children's ranges (reducing their boxes), or
// copy of a finished leaf's particles to the tree's output arrays.  One block per chunk
// (chunks beyond the grid in turn); chunks with node -1 were reserved and not used.
__global__ void k_scatter(const BChunk* __restrict__ chunks, BNode* nodes,
                          const uint8_t* __restrict__ oct, const double* __restrict__ ax,
                          const double* __restrict__ ay, const double* __restrict__ az,
                          const double* __restrict__ aq, const int32_t* __restrict__ ai,
                          double* bx, double* by, double* bz, double* bq, int32_t* bi,
                          double* ox, double* oy, double* oz, double* oq, int32_t* oi,
                          bool has_q, int64_t nck, const int32_t* dlv) {
    __shared__ int wcnt[kThreads / 32][8];
    __shared__ int run[8];
    __shared__ unsigned long long box[8][6];
    __shared__ int pre[8], obase[8];
    if (dlv) nck = dlv[2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c = blockIdx.x; c < nck; c += gridDim.x) {
        const BChunk ch = chunks[c];
        if (ch.node < 0) continue;
        BNode& nd = nodes[ch.node];
        if (nd.split == 0) {
            for (int32_t i = ch.start + threadIdx.x; i < ch.end; i += blockDim.x) {
                ox[i] = ax[i];
                oy[i] = ay[i];
                oz[i] = az[i];
                if (has_q) oq[i] = aq[i];
                oi[i] = ai[i];
            }
            continue;
        }
        __syncthreads();   // the previous chunk's shared state is no longer read
        if (threadIdx.x < 8) {
            run[threadIdx.x] = 0;
            pre[threadIdx.x] = ch.prefix[threadIdx.x];
            obase[threadIdx.x] = nd.octbase[threadIdx.x];
        }
        if (threadIdx.x < 48) box[threadIdx.x / 6][threadIdx.x % 6] = (threadIdx.x % 6) < 3 ? ~0ULL : 0ULL;
        __syncthreads();
        for (int32_t t0 = ch.start; t0 < ch.end; t0 += kThreads) {
            const int32_t i = t0 + threadIdx.x;
            const bool in = i < ch.end;
            const int o = in ? oct[i] : 8;
            const unsigned same = __match_any_sync(0xffffffffu, o);
            const int rank = __popc(same & ((1u << lane) - 1u));
            if (threadIdx.x < kThreads / 32 * 8) wcnt[threadIdx.x >> 3][threadIdx.x & 7] = 0;
            __syncthreads();
            if (in && rank == 0) wcnt[warp][o] = __popc(same);
            __syncthreads();
            if (in) {
                int before = 0;
                for (int w = 0; w < warp; ++w) before += wcnt[w][o];
                const int32_t dst = obase[o] + pre[o] + run[o] + before + rank;
                const double vx = ax[i], vy = ay[i], vz = az[i];
                bx[dst] = vx;
                by[dst] = vy;
                bz[dst] = vz;
                if (has_q) bq[dst] = aq[i];
                bi[dst] = ai[i];
                atomicMin(&box[o][0], okey(vx));
                atomicMin(&box[o][1], okey(vy));
                atomicMin(&box[o][2], okey(vz));
                atomicMax(&box[o][3], okey(vx));
                atomicMax(&box[o][4], okey(vy));
                atomicMax(&box[o][5], okey(vz));
            }
            __syncthreads();
            if (threadIdx.x < 8) {
                int s = 0;
                for (int w = 0; w < kThreads / 32; ++w) s += wcnt[w][threadIdx.x];
                run[threadIdx.x] += s;
            }
            __syncthreads();
        }
        if (threadIdx.x < 48) {
            const int o = threadIdx.x / 6, d = threadIdx.x % 6;
            const int id = nd.octchild[o];
            if (id >= 0 && run[o] > 0) {
                if (d < 3)
                    atomicMin(&nodes[id].key[d], box[o][d]);
                else
                    atomicMax(&nodes[id].key[d], box[o][d]);
            }
        }
    }
}

// Sized on the device: the range and chunk count of the next level ({first, end, chunks} at
// dlv[3..5]) from the level just split and the two counters.
__global__ void k_level_advance(int32_t* dlv, const int32_t* counters) {
    dlv[3] = dlv[1];
    dlv[4] = counters[0];
    dlv[5] = counters[1];
}

__global__ void k_subtree_size(BNode* nodes, int32_t l0, int32_t l1, const int32_t* dlv) {
    if (dlv) {
        l0 = dlv[0];
        l1 = dlv[1];
    }
    for (int64_t v = l0 + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < l1;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        BNode& nd = nodes[v];
        int s = 1;
        for (int c = 0; c < nd.nch; ++c) s += nodes[nd.child[c]].size;
        nd.size = s;
    }
}

__global__ void k_dfs_ids(BNode* nodes, int32_t l0, int32_t l1, const int32_t* dlv) {
    if (dlv) {
        l0 = dlv[0];
        l1 = dlv[1];
    }
    for (int64_t v = l0 + static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < l1;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const BNode& nd = nodes[v];
        int d = nd.dfs + 1;
        for (int c = 0; c < nd.nch; ++c) {
            nodes[nd.child[c]].dfs = d;
            d += nodes[nd.child[c]].size;
        }
    }
}

// Node arrays in DFS order.  Sized on the device the node count comes from *dm and the
// entries from it up to `cap` are written as inert nodes (level -1, no particles, no children).
__global__ void k_emit(const BNode* __restrict__ nodes, int32_t m, int32_t* begin,
                       int32_t* count, int32_t* parent, int32_t* level, int32_t* nch,
                       int32_t* child, double* lo, double* hi, double* center, double* radius,
                       int32_t* is_leaf, const int32_t* dm, int32_t cap) {
    if (dm) m = *dm;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < cap;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (v >= m) {
            begin[v] = 0;
            count[v] = 0;
            parent[v] = -1;
            level[v] = -1;
            nch[v] = 0;
            for (int c = 0; c < 8; ++c) child[8 * v + c] = -1;
            for (int k = 0; k < 3; ++k) lo[3 * v + k] = hi[3 * v + k] = center[3 * v + k] = 0.0;
            radius[v] = 0.0;
            is_leaf[v] = 0;
            continue;
        }
        const BNode& nd = nodes[v];
        const int32_t d = nd.dfs;
        begin[d] = nd.begin;
        count[d] = nd.count;
        parent[d] = nd.parent >= 0 ? nodes[nd.parent].dfs : -1;
        level[d] = nd.level;
        nch[d] = nd.nch;
        for (int c = 0; c < 8; ++c) child[8 * d + c] = c < nd.nch ? nodes[nd.child[c]].dfs : -1;
        for (int k = 0; k < 3; ++k) {
            lo[3 * d + k] = nd.lo[k];
            hi[3 * d + k] = nd.hi[k];
            center[3 * d + k] = nd.center[k];
        }
        radius[d] = nd.radius;
        is_leaf[d] = nd.nch == 0 ? 1 : 0;
    }
}

__global__ void k_level_init(int32_t* dlv, int32_t end, int32_t nck) {
    dlv[0] = 0;
    dlv[1] = end;
    dlv[2] = nck;
}

// Non-finite input raises bit 1 of the flag of a build sized on the device.
__global__ void k_input_flag(const int32_t* bad, int32_t* flag) {
    if (*bad) atomicOr(flag, 2);
}

__global__ void k_leaf_list(const int32_t* __restrict__ is_leaf,
                            const int32_t* __restrict__ pos, int32_t m, int32_t* leaves) {
    int32_t v = static_cast<int32_t>(blockIdx.x * blockDim.x + threadIdx.x);
    if (v < m && is_leaf[v]) leaves[pos[v]] = v;
}

}  // namespace

// Sized on the device (caps != nullptr): buffers at the capacities, a fixed number of level
// iterations whose ranges stay in device memory (a level with no nodes costs empty launches),
// and no host synchronisation, so the build can be captured in a graph.  The tree equals the
// host-driven build's whenever the flag stays 0: the kernels and their order are the same,
// only the launch grids differ.
static void build_tree_sized(Context* ctx, const double* x, const double* y, const double* z,
                             const double* q, int32_t n, int32_t max_leaf, Tree* out,
                             const Caps& caps, DBuf<double> (&A)[4], DBuf<double> (&B)[4],
                             DBuf<int32_t>& Ai, DBuf<int32_t>& Bi) {
    cudaStream_t s = ctx->stream;
    const bool has_q = q != nullptr;
    require(caps.nodes >= 1 && caps.levels >= 1 && caps.level_nodes >= 1 && caps.chunks >= 1,
            "tree: capacities must be positive");
    const int64_t root_chunks = ceil_div(n, kCh);
    const int64_t chunk_cap = std::max<int64_t>(caps.chunks, root_chunks);
    const int Lc = caps.levels;
    DBuf<uint8_t> oct(ctx, n);
    DBuf<int32_t> counters(ctx, 4);
    DBuf<BNode> nodes(ctx, caps.nodes);
    DBuf<BChunk> chunks[2] = {DBuf<BChunk>(ctx, chunk_cap), DBuf<BChunk>(ctx, chunk_cap)};
    DBuf<int32_t> lv(ctx, 3 * (Lc + 1));       // per level: first node, end node, chunks
    const int32_t first[3] = {0, 1, static_cast<int32_t>(root_chunks)};
    k_root_init<<<1, 1, 0, s>>>(nodes.p, n, counters.p); ++ctx->launches;
    k_level_init<<<1, 1, 0, s>>>(lv.p, first[1], first[2]); ++ctx->launches;
    k_root_chunks<<<grid_for(root_chunks, kThreads), kThreads, 0, s>>>(chunks[0].p, n); ++ctx->launches;
    {
        const unsigned g = std::min<unsigned>(grid_for(n, kThreads), 8u * std::max(1, ctx->sm_count));
        k_root_copy<<<g, kThreads, 0, s>>>(x, y, z, q, n, A[0].p, A[1].p, A[2].p, A[3].p, Ai.p,
                                           nodes.p, counters.p + 2); ++ctx->launches;
    }
    BLTC_LAUNCH_CHECK("tree root");
    const unsigned gn = grid_for(caps.level_nodes, kThreads);
    const unsigned gb = static_cast<unsigned>(std::min<int64_t>(caps.level_nodes, 4 * std::max(1, ctx->sm_count)));
    const unsigned gc = static_cast<unsigned>(std::min<int64_t>(chunk_cap, 8 * std::max(1, ctx->sm_count)));
    int cur = 0;
    for (int lvl = 0; lvl < Lc; ++lvl) {
        const int nxt = cur ^ 1;
        int32_t* dlv = lv.p + 3 * lvl;
        BLTC_CUDA(cudaMemsetAsync(counters.p + 1, 0, sizeof(int32_t), s));   // next chunk
        k_node_prepare<<<gn, kThreads, 0, s>>>(nodes.p, 0, 0, max_leaf, dlv, caps.flag, lvl == Lc - 1); ++ctx->launches;
        k_classify<<<gc, kThreads, 0, s>>>(chunks[cur].p, nodes.p, A[0].p, A[1].p, A[2].p, oct.p, 0, dlv); ++ctx->launches;
        k_node_split<<<gb, kThreads, 0, s>>>(nodes.p, 0, 0, chunks[cur].p, chunks[nxt].p, counters.p, dlv,
                                             caps.nodes, chunk_cap, caps.flag); ++ctx->launches;
        k_scatter<<<gc, kThreads, 0, s>>>(
            chunks[cur].p, nodes.p, oct.p, A[0].p, A[1].p, A[2].p, A[3].p, Ai.p, B[0].p, B[1].p,
            B[2].p, B[3].p, Bi.p, out->px.p, out->py.p, out->pz.p, has_q ? out->pq.p : nullptr,
            out->perm.p, has_q, 0, dlv); ++ctx->launches;
        k_level_advance<<<1, 1, 0, s>>>(dlv, counters.p); ++ctx->launches;
        BLTC_LAUNCH_CHECK("tree level");
        for (int k = 0; k < 4; ++k) std::swap(A[k], B[k]);
        std::swap(Ai, Bi);
        cur = nxt;
    }
    // non-finite input: the host-driven build reports it; here it raises the flag (bit 1)
    k_input_flag<<<1, 1, 0, s>>>(counters.p + 2, caps.flag); ++ctx->launches;
    for (int lvl = Lc - 1; lvl >= 0; --lvl) {
        k_subtree_size<<<gn, kThreads, 0, s>>>(nodes.p, 0, 0, lv.p + 3 * lvl); ++ctx->launches;
    }
    BLTC_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(nodes.p) + offsetof(BNode, dfs), 0,
                              sizeof(int32_t), s));
    for (int lvl = 0; lvl < Lc; ++lvl) {
        k_dfs_ids<<<gn, kThreads, 0, s>>>(nodes.p, 0, 0, lv.p + 3 * lvl); ++ctx->launches;
    }
    const int32_t m = caps.nodes;
    out->n_nodes = m;
    out->n_levels = Lc;
    out->caps = &caps;
    out->dcount = DBuf<int32_t>(ctx, 2);
    out->begin = DBuf<int32_t>(ctx, m);
    out->count = DBuf<int32_t>(ctx, m);
    out->parent = DBuf<int32_t>(ctx, m);
    out->level = DBuf<int32_t>(ctx, m);
    out->nch = DBuf<int32_t>(ctx, m);
    out->child = DBuf<int32_t>(ctx, 8 * static_cast<int64_t>(m));
    out->lo = DBuf<double>(ctx, 3 * static_cast<int64_t>(m));
    out->hi = DBuf<double>(ctx, 3 * static_cast<int64_t>(m));
    out->center = DBuf<double>(ctx, 3 * static_cast<int64_t>(m));
    out->radius = DBuf<double>(ctx, m);
    DBuf<int32_t> is_leaf(ctx, m), pos(ctx, m);
    BLTC_CUDA(cudaMemcpyAsync(out->dcount.p, counters.p, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    k_emit<<<grid_for(m, kThreads, 8 * std::max(1, ctx->sm_count)), kThreads, 0, s>>>(
        nodes.p, 0, out->begin.p, out->count.p, out->parent.p, out->level.p, out->nch.p,
        out->child.p, out->lo.p, out->hi.p, out->center.p, out->radius.p, is_leaf.p, counters.p, m); ++ctx->launches;
    BLTC_LAUNCH_CHECK("tree emit");
    exclusive_scan_i32(ctx, is_leaf.p, pos.p, m, out->dcount.p + 1);
    out->n_leaves = m;
    out->leaves = DBuf<int32_t>(ctx, m);
    BLTC_CUDA(cudaMemsetAsync(out->leaves.p, 0xff, sizeof(int32_t) * m, s));   // -1: no batch
    k_leaf_list<<<grid_for(m, kThreads), kThreads, 0, s>>>(is_leaf.p, pos.p, m, out->leaves.p); ++ctx->launches;
    BLTC_LAUNCH_CHECK("tree leaves");
}

void build_tree(Context* ctx, const double* x, const double* y, const double* z,
                const double* q, int64_t n64, int32_t max_leaf, Tree* out, const Caps* caps) {
    require(n64 >= 1 && n64 < (int64_t(1) << 31), "tree: n must be in [1, 2^31)");
    require(max_leaf >= 1, "tree: max_leaf must be >= 1");
    require(x && y && z, "tree: NULL coordinate pointer");
    const int32_t n = static_cast<int32_t>(n64);
    const bool has_q = q != nullptr;
    cudaStream_t s = ctx->stream;

    out->ctx = ctx;
    out->n = n;
    out->max_leaf = max_leaf;
    out->has_q = has_q;
    out->px = DBuf<double>(ctx, n);
    out->py = DBuf<double>(ctx, n);
    out->pz = DBuf<double>(ctx, n);
    if (has_q) out->pq = DBuf<double>(ctx, n);
    out->perm = DBuf<int32_t>(ctx, n);

    DBuf<double> A[4] = {DBuf<double>(ctx, n), DBuf<double>(ctx, n), DBuf<double>(ctx, n),
                         DBuf<double>(ctx, has_q ? n : 1)};
    DBuf<double> B[4] = {DBuf<double>(ctx, n), DBuf<double>(ctx, n), DBuf<double>(ctx, n),
                         DBuf<double>(ctx, has_q ? n : 1)};
    DBuf<int32_t> Ai(ctx, n), Bi(ctx, n);
    if (caps) {
        build_tree_sized(ctx, x, y, z, q, n, max_leaf, out, *caps, A, B, Ai, Bi);
        return;
    }
    DBuf<uint8_t> oct(ctx, n);
    DBuf<int32_t> counters(ctx, 4);   // next node, next chunk, bad-input flag
    DBuf<int32_t> unused_flag(ctx, 1);
    const int64_t root_chunks = ceil_div(n, kCh);

    int64_t node_cap = std::max<int64_t>(64, 4 * ceil_div(n, std::max(1, max_leaf)) + 64);
    DBuf<BNode> nodes(ctx, node_cap);
    int64_t chunk_cap[2] = {root_chunks + 64, root_chunks + 64};
    DBuf<BChunk> chunks[2] = {DBuf<BChunk>(ctx, chunk_cap[0]), DBuf<BChunk>(ctx, chunk_cap[1])};

    k_root_init<<<1, 1, 0, s>>>(nodes.p, n, counters.p); ++ctx->launches;
    k_root_chunks<<<grid_for(root_chunks, kThreads), kThreads, 0, s>>>(chunks[0].p, n); ++ctx->launches;
    {
        const unsigned g = std::min<unsigned>(grid_for(n, kThreads), 8u * std::max(1, ctx->sm_count));
        k_root_copy<<<g, kThreads, 0, s>>>(x, y, z, q, n, A[0].p, A[1].p, A[2].p, A[3].p, Ai.p,
                                           nodes.p, counters.p + 2); ++ctx->launches;
    }
    BLTC_LAUNCH_CHECK("tree root");

    std::vector<int32_t> level_start = {0, 1};
    int cur = 0;                   // chunk buffer of the current level
    int64_t n_chunks = root_chunks;
    int32_t next_node = 1;
    bool checked_input = false;
    for (int lvl = 0;; ++lvl) {
        const int32_t l0 = level_start[lvl], l1 = level_start[lvl + 1];
        const int32_t nl = l1 - l0;
        // room for up to 8 children per node of this level
        const int64_t need_nodes = static_cast<int64_t>(l1) + 8 * static_cast<int64_t>(nl);
        if (need_nodes > node_cap) {
            int64_t cap = std::max(need_nodes, 2 * node_cap);
            DBuf<BNode> bigger(ctx, cap);
            BLTC_CUDA(cudaMemcpyAsync(bigger.p, nodes.p, sizeof(BNode) * l1,
                                      cudaMemcpyDeviceToDevice, s));
            nodes = std::move(bigger);
            node_cap = cap;
        }
        const int nxt = cur ^ 1;
        const int64_t need_chunks = root_chunks + 8 * static_cast<int64_t>(nl) + 1;
        if (need_chunks > chunk_cap[nxt]) {
            chunk_cap[nxt] = std::max(need_chunks, 2 * chunk_cap[nxt]);
            chunks[nxt] = DBuf<BChunk>(ctx, chunk_cap[nxt]);
        }
        BLTC_CUDA(cudaMemsetAsync(counters.p + 1, 0, sizeof(int32_t), s));   // next chunk

        k_node_prepare<<<grid_for(nl, kThreads), kThreads, 0, s>>>(nodes.p, l0, l1, max_leaf, nullptr,
                                                                   nullptr, false); ++ctx->launches;
        k_classify<<<static_cast<unsigned>(n_chunks), kThreads, 0, s>>>(
            chunks[cur].p, nodes.p, A[0].p, A[1].p, A[2].p, oct.p, n_chunks, nullptr); ++ctx->launches;
        // the capacities were made sufficient above: no reservation can fail
        k_node_split<<<static_cast<unsigned>(nl), kThreads, 0, s>>>(nodes.p, l0, l1, chunks[cur].p,
                                                                   chunks[nxt].p, counters.p, nullptr,
                                                                   node_cap, chunk_cap[nxt],
                                                                   unused_flag.p); ++ctx->launches;
        k_scatter<<<static_cast<unsigned>(n_chunks), kThreads, 0, s>>>(
            chunks[cur].p, nodes.p, oct.p, A[0].p, A[1].p, A[2].p, A[3].p, Ai.p, B[0].p, B[1].p,
            B[2].p, B[3].p, Bi.p, out->px.p, out->py.p, out->pz.p, has_q ? out->pq.p : nullptr,
            out->perm.p, has_q, n_chunks, nullptr); ++ctx->launches;
        BLTC_LAUNCH_CHECK("tree level");
        const int64_t* w = ctx->read_words(counters.p, 2);   // int32 x4 packed in 2 words
        const int32_t* c32 = reinterpret_cast<const int32_t*>(w);
        if (!checked_input) {
            require(c32[2] == 0, "tree: non-finite coordinate or charge");
            checked_input = true;
        }
        const int32_t made = c32[0];
        const int32_t nchk = c32[1];
        if (made == next_node) break;      // no node of this level split
        next_node = made;
        level_start.push_back(made);
        for (int k = 0; k < 4; ++k) std::swap(A[k], B[k]);
        std::swap(Ai, Bi);
        cur = nxt;
        n_chunks = nchk;
    }

    const int32_t m = next_node;
    const int n_levels = static_cast<int>(level_start.size()) - 1;
    for (int lvl = n_levels - 1; lvl >= 0; --lvl) {
        const int32_t l0 = level_start[lvl], l1 = level_start[lvl + 1];
        k_subtree_size<<<grid_for(l1 - l0, kThreads), kThreads, 0, s>>>(nodes.p, l0, l1, nullptr); ++ctx->launches;
    }
    BLTC_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(nodes.p) + offsetof(BNode, dfs), 0,
                              sizeof(int32_t), s));
    for (int lvl = 0; lvl < n_levels; ++lvl) {
        const int32_t l0 = level_start[lvl], l1 = level_start[lvl + 1];
        k_dfs_ids<<<grid_for(l1 - l0, kThreads), kThreads, 0, s>>>(nodes.p, l0, l1, nullptr); ++ctx->launches;
    }
    out->n_nodes = m;
    out->n_levels = n_levels;
    out->begin = DBuf<int32_t>(ctx, m);
    out->count = DBuf<int32_t>(ctx, m);
    out->parent = DBuf<int32_t>(ctx, m);
    out->level = DBuf<int32_t>(ctx, m);
    out->nch = DBuf<int32_t>(ctx, m);
    out->child = DBuf<int32_t>(ctx, 8 * static_cast<int64_t>(m));
    out->lo = DBuf<double>(ctx, 3 * static_cast<int64_t>(m));
    out->hi = DBuf<double>(ctx, 3 * static_cast<int64_t>(m));
    out->center = DBuf<double>(ctx, 3 * static_cast<int64_t>(m));
    out->radius = DBuf<double>(ctx, m);
    DBuf<int32_t> is_leaf(ctx, m), pos(ctx, m), n_leaf(ctx, 1);
    k_emit<<<grid_for(m, kThreads), kThreads, 0, s>>>(
        nodes.p, m, out->begin.p, out->count.p, out->parent.p, out->level.p, out->nch.p,
        out->child.p, out->lo.p, out->hi.p, out->center.p, out->radius.p, is_leaf.p, nullptr, m); ++ctx->launches;
    BLTC_LAUNCH_CHECK("tree emit");
    exclusive_scan_i32(ctx, is_leaf.p, pos.p, m, n_leaf.p);
    const int32_t nleaves = *reinterpret_cast<const int32_t*>(ctx->read_words(n_leaf.p, 1));
    out->n_leaves = nleaves;
    out->leaves = DBuf<int32_t>(ctx, nleaves);
    k_leaf_list<<<grid_for(m, kThreads), kThreads, 0, s>>>(is_leaf.p, pos.p, m, out->leaves.p); ++ctx->launches;
    BLTC_LAUNCH_CHECK("tree leaves");
}

void tree_counts(Context* ctx, const Tree& t, Caps* caps) {
    const int64_t m = t.n_nodes;
    std::vector<int32_t> level(static_cast<size_t>(m)), count(static_cast<size_t>(m));
    BLTC_CUDA(cudaMemcpyAsync(level.data(), t.level.p, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, ctx->stream));
    BLTC_CUDA(cudaMemcpyAsync(count.data(), t.count.p, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, ctx->stream));
    BLTC_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<int64_t> nodes_at(static_cast<size_t>(t.n_levels) + 1, 0), chunks_at(nodes_at.size(), 0);
    for (int64_t v = 0; v < m; ++v) {
        const size_t L = static_cast<size_t>(level[static_cast<size_t>(v)]);
        nodes_at[L] += 1;
        chunks_at[L] += ceil_div(count[static_cast<size_t>(v)], kCh);
    }
    caps->nodes = static_cast<int32_t>(m);
    caps->levels = t.n_levels;
    caps->level_nodes = static_cast<int32_t>(*std::max_element(nodes_at.begin(), nodes_at.end()));
    caps->chunks = *std::max_element(chunks_at.begin(), chunks_at.end());
}

}  // namespace bltc
