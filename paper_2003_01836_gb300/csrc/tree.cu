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

// (1) Box, centre, radius and split of every node of the level.
__global__ void k_node_prepare(BNode* nodes, int32_t l0, int32_t l1, int32_t max_leaf) {
    int32_t v = l0 + static_cast<int32_t>(blockIdx.x * blockDim.x + threadIdx.x);
    if (v >= l1) return;
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
    nd.split = split;
}

// (2) Octant of every particle of a splitting node, and the chunk's histogram.
__global__ void k_classify(BChunk* chunks, const BNode* __restrict__ nodes,
                           const double* __restrict__ ax, const double* __restrict__ ay,
                           const double* __restrict__ az, uint8_t* __restrict__ oct) {
    __shared__ int hist[8];
    const BChunk ch = chunks[blockIdx.x];
    const BNode& nd = nodes[ch.node];
    const int split = nd.split;
    if (split == 0) return;
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
    if (threadIdx.x < 8) chunks[blockIdx.x].hist[threadIdx.x] = hist[threadIdx.x];
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
// creation of the children (ids and chunk ranges from two atomic counters).
__global__ void k_node_split(BNode* nodes, int32_t l0, BChunk* chunks, BChunk* next_chunks,
                             int32_t* counters /* [0] next node, [1] next chunk */) {
    __shared__ int ws[kThreads / 32];
    __shared__ int tot[8];
    __shared__ int base_id, base_chunk[8];
    BNode& nd = nodes[l0 + blockIdx.x];
    if (nd.split == 0) return;
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
        for (int o = 0; o < 8; ++o) {
            tot[o] = carry[o];
            nonempty += carry[o] > 0;
        }
        if (nonempty <= 1) {
            nd.split = 0;     // the split separates nothing: the node stays a leaf
            base_id = -1;
        } else {
            nd.nch = nonempty;
            base_id = atomicAdd(&counters[0], nonempty);
            int pos = nd.begin, c = 0;
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
                    k.parent = l0 + static_cast<int32_t>(blockIdx.x);
                    k.level = nd.level + 1;
                    k.nch = 0;
                    k.split = 0;
                    k.nchunk = (tot[o] + kCh - 1) / kCh;
                    k.chunk0 = atomicAdd(&counters[1], k.nchunk);
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
    __syncthreads();
    if (base_id < 0) return;
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

// (4) Stable scatter of each chunk into its children's ranges (reducing their boxes), or
// copy of a finished leaf's particles to the tree's output arrays.
__global__ void k_scatter(const BChunk* __restrict__ chunks, BNode* nodes,
                          const uint8_t* __restrict__ oct, const double* __restrict__ ax,
                          const double* __restrict__ ay, const double* __restrict__ az,
                          const double* __restrict__ aq, const int32_t* __restrict__ ai,
                          double* bx, double* by, double* bz, double* bq, int32_t* bi,
                          double* ox, double* oy, double* oz, double* oq, int32_t* oi,
                          bool has_q) {
    __shared__ int wcnt[kThreads / 32][8];
    __shared__ int run[8];
    __shared__ unsigned long long box[8][6];
    __shared__ int pre[8], obase[8];
    const BChunk ch = chunks[blockIdx.x];
    BNode& nd = nodes[ch.node];
    if (nd.split == 0) {
        for (int32_t i = ch.start + threadIdx.x; i < ch.end; i += blockDim.x) {
            ox[i] = ax[i];
            oy[i] = ay[i];
            oz[i] = az[i];
            if (has_q) oq[i] = aq[i];
            oi[i] = ai[i];
        }
        return;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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

__global__ void k_subtree_size(BNode* nodes, int32_t l0, int32_t l1) {
    int32_t v = l0 + static_cast<int32_t>(blockIdx.x * blockDim.x + threadIdx.x);
    if (v >= l1) return;
    BNode& nd = nodes[v];
    int s = 1;
    for (int c = 0; c < nd.nch; ++c) s += nodes[nd.child[c]].size;
    nd.size = s;
}

__global__ void k_dfs_ids(BNode* nodes, int32_t l0, int32_t l1) {
    int32_t v = l0 + static_cast<int32_t>(blockIdx.x * blockDim.x + threadIdx.x);
    if (v >= l1) return;
    const BNode& nd = nodes[v];
    int d = nd.dfs + 1;
    for (int c = 0; c < nd.nch; ++c) {
        nodes[nd.child[c]].dfs = d;
        d += nodes[nd.child[c]].size;
    }
}

__global__ void k_emit(const BNode* __restrict__ nodes, int32_t m, int32_t* begin,
                       int32_t* count, int32_t* parent, int32_t* level, int32_t* nch,
                       int32_t* child, double* lo, double* hi, double* center, double* radius,
                       int32_t* is_leaf) {
    int32_t v = static_cast<int32_t>(blockIdx.x * blockDim.x + threadIdx.x);
    if (v >= m) return;
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

__global__ void k_leaf_list(const int32_t* __restrict__ is_leaf,
                            const int32_t* __restrict__ pos, int32_t m, int32_t* leaves) {
    int32_t v = static_cast<int32_t>(blockIdx.x * blockDim.x + threadIdx.x);
    if (v < m && is_leaf[v]) leaves[pos[v]] = v;
}

}  // namespace

void build_tree(Context* ctx, const double* x, const double* y, const double* z,
                const double* q, int64_t n64, int32_t max_leaf, Tree* out) {
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
    DBuf<uint8_t> oct(ctx, n);
    DBuf<int32_t> counters(ctx, 4);   // next node, next chunk, bad-input flag
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

        k_node_prepare<<<grid_for(nl, kThreads), kThreads, 0, s>>>(nodes.p, l0, l1, max_leaf); ++ctx->launches;
        k_classify<<<static_cast<unsigned>(n_chunks), kThreads, 0, s>>>(
            chunks[cur].p, nodes.p, A[0].p, A[1].p, A[2].p, oct.p); ++ctx->launches;
        k_node_split<<<static_cast<unsigned>(nl), kThreads, 0, s>>>(nodes.p, l0, chunks[cur].p,
                                                                   chunks[nxt].p, counters.p); ++ctx->launches;
        k_scatter<<<static_cast<unsigned>(n_chunks), kThreads, 0, s>>>(
            chunks[cur].p, nodes.p, oct.p, A[0].p, A[1].p, A[2].p, A[3].p, Ai.p, B[0].p, B[1].p,
            B[2].p, B[3].p, Bi.p, out->px.p, out->py.p, out->pz.p, has_q ? out->pq.p : nullptr,
            out->perm.p, has_q); ++ctx->launches;
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
        k_subtree_size<<<grid_for(l1 - l0, kThreads), kThreads, 0, s>>>(nodes.p, l0, l1); ++ctx->launches;
    }
    BLTC_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(nodes.p) + offsetof(BNode, dfs), 0,
                              sizeof(int32_t), s));
    for (int lvl = 0; lvl < n_levels; ++lvl) {
        const int32_t l0 = level_start[lvl], l1 = level_start[lvl + 1];
        k_dfs_ids<<<grid_for(l1 - l0, kThreads), kThreads, 0, s>>>(nodes.p, l0, l1); ++ctx->launches;
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
        out->child.p, out->lo.p, out->hi.p, out->center.p, out->radius.p, is_leaf.p); ++ctx->launches;
    BLTC_LAUNCH_CHECK("tree emit");
    exclusive_scan_i32(ctx, is_leaf.p, pos.p, m, n_leaf.p);
    const int32_t nleaves = *reinterpret_cast<const int32_t*>(ctx->read_words(n_leaf.p, 1));
    out->n_leaves = nleaves;
    out->leaves = DBuf<int32_t>(ctx, nleaves);
    k_leaf_list<<<grid_for(m, kThreads), kThreads, 0, s>>>(is_leaf.p, pos.p, m, out->leaves.p); ++ctx->launches;
    BLTC_LAUNCH_CHECK("tree leaves");
}

}  // namespace bltc
