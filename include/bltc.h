/*
 * bltc.h -- C ABI of the GB300 barycentric Lagrange treecode (BLTC) library.
 *
 * The library evaluates the potentials
 *     phi(x_i) = sum_j G(x_i, y_j) q_j,   G = 1/r (Coulomb) or exp(-kappa r)/r (Yukawa)
 * of Eq. 1-2 of Vaughn, Wilson and Krasny, "A GPU-Accelerated Barycentric Lagrange
 * Treecode" (2020), with the treecode of Algorithm 1: a tree of source clusters and target
 * batches (Sec. II-D), interaction lists from the multipole acceptance criterion (MAC,
 * Eq. 13), modified charges at tensor-product Chebyshev points (Eq. 12, Sec. II-C), and the
 * batch-cluster approximation (Eq. 11) and direct (Eq. 9) sums.  Every step runs on the GPU.
 *
 * Conventions, for every entry point unless its comment says otherwise:
 *   - Pointers named x, y, z, q, phi, tx, ... are DEVICE pointers owned by the caller
 *     (for example torch tensors' data_ptr()), FP64, contiguous, one value per particle in
 *     the caller's order.  The library never frees them and keeps them past the call only
 *     where the entry point says so (bltc_graph_create binds q and phi to the graph).
 *   - Work is enqueued on the context's stream (bltc_context_set_stream) and may still be
 *     running when the call returns.  Calls whose comment says "synchronizes" wait for the
 *     stream before returning.  A call that needs a count computed on the device (tree
 *     build, list build, evaluate, solve) synchronizes the stream internally.
 *   - Handles (bltc_tree, bltc_lists, bltc_graph) own their device memory, allocated through the
 *     context's allocator; only the matching *_destroy frees it.  A handle must not
 *     outlive its context.
 *   - Every call returns a bltc_status; on failure nothing observable was written to the
 *     caller's output buffers, and bltc_last_error() describes the failure.  No C++
 *     exception crosses this boundary.
 *   - A context is not thread-safe: use one per host thread.
 *
 * Readings of the paper that the library implements exactly (shared with the test oracle,
 * which is a separate implementation):
 *   - a pair with r^2 == 0 is skipped (targets are the sources, Eq. 1);
 *   - boxes are the minimal axis-aligned boxes of their particles (Sec. II-D), -0.0 < +0.0;
 *   - centre c = 0.5*(lo+hi), radius = |0.5*(hi-lo)|, R = |c_B - c_C|, all FP64, no fused
 *     multiply-add; the MAC's geometric part is (r_B + r_C)/R < theta (a NaN ratio fails);
 *   - dimension d is split iff (hi_d-lo_d)*sqrt(2) >= longest extent (Sec. III-A); a
 *     particle goes low iff coord < 0.5*(lo_d+hi_d); children in increasing octant order
 *     (bit0/1/2 = x/y/z high), empty ones dropped, stable partition; a node is a leaf iff
 *     count <= max_leaf, its extent is zero, or the split leaves one non-empty child; node
 *     ids are DFS pre-order;
 *   - Chebyshev points s_k = lo + 0.5*(cos(pi k/n)+1)*(hi-lo) with s_0 = hi, s_n = lo;
 *     a source coordinate within DBL_MIN of s_k takes L_k = 1 exactly (Sec. II-C).
 */
#ifndef BLTC_H
#define BLTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BLTC_VERSION 1
#define BLTC_MAX_DEGREE 16

typedef enum bltc_status {
    BLTC_OK = 0,
    BLTC_ERR_ARG = -1,      /* an argument is out of range or non-finite; nothing was run */
    BLTC_ERR_OOM = -2,      /* the allocator returned no memory */
    BLTC_ERR_CUDA = -3,     /* a CUDA call failed; the message names it */
    BLTC_ERR_TIMEOUT = -4,  /* reserved for bounded device-side waits (none in this version) */
    BLTC_ERR_STATE = -5,    /* handles that do not belong together, or a step missing */
    BLTC_ERR_CANCELLED = -6 /* a served request was cancelled before admission */
} bltc_status;

enum { BLTC_KERNEL_COULOMB = 0, BLTC_KERNEL_YUKAWA = 1 };
/* Ids of user kernels registered in a context (bltc_kernel_register) start here. */
#define BLTC_KERNEL_USER_BASE 16

/* FP64: every step in FP64 (the reference path; Sec. IV computes in double precision).
 * MIXED: kernel evaluations in FP32 on coordinates relative to the batch centre with FP32
 * sums over one cluster; cross-cluster sums, boxes, MAC, Chebyshev points and the
 * source-minus-point differences of the modified charges stay FP64. */
enum { BLTC_PRECISION_FP64 = 0, BLTC_PRECISION_MIXED = 1 };

/* Treecode parameters of Algorithm 1 ("input: theta, n, N_L, N_B") plus the kernel. */
typedef struct bltc_params {
    int32_t degree;      /* n, interpolation degree, 1..BLTC_MAX_DEGREE; (n+1)^3 points */
    int32_t leaf_size;   /* N_L >= 1, source clusters hold at most N_L particles */
    int32_t batch_size;  /* N_B >= 1, target batches hold at most N_B particles */
    int32_t kernel;      /* BLTC_KERNEL_COULOMB, BLTC_KERNEL_YUKAWA or a registered user id */
    int32_t precision;   /* BLTC_PRECISION_FP64 or BLTC_PRECISION_MIXED */
    int32_t tile;        /* the mixed sweep's tile shape, 0 for the defaults (bltc_autotune_tile
                          * chooses one): bits 0-3 cap the source groups of a batch (0: 8;
                          * else 1, 2, 4 or 8 thread groups of 256/G threads that split a
                          * batch's sources, each covering the batch in passes of 2048/G
                          * targets), bits 4-11 the work items per resident block of the
                          * persistent sweep (0: 16; else 1..255; the item size follows), the
                          * other bits 0.  The shape fixes the summation order, not the
                          * arithmetic: results differ by rounding only. */
    double theta;        /* MAC parameter, 0 <= theta < 1 (theta = 0: all direct) */
    double kappa;        /* Yukawa inverse Debye length, >= 0 (ignored for Coulomb); the
                          * parameter of a user kernel */
} bltc_params;

typedef struct bltc_context bltc_context;
typedef struct bltc_tree bltc_tree;
typedef struct bltc_lists bltc_lists;
typedef struct bltc_graph bltc_graph;

/* Optional allocator hooks.  alloc returns device memory of >= bytes usable in stream order
 * on `stream`, or NULL; free releases it in stream order.  Default: a CUDA memory pool of
 * the context's device (cudaMallocFromPoolAsync / cudaFreeAsync). */
typedef void* (*bltc_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*bltc_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* ---- context ---------------------------------------------------------------------- */

/* Creates a context on CUDA `device` enqueuing on `stream` (a cudaStream_t; NULL = the
 * legacy default stream).  *out receives the handle.  Errors: ARG (out NULL, bad device),
 * CUDA. */
bltc_status bltc_context_create(int device, void* stream, bltc_context** out);
void bltc_context_destroy(bltc_context* ctx);
bltc_status bltc_context_set_stream(bltc_context* ctx, void* stream);
bltc_status bltc_context_set_allocator(bltc_context* ctx, bltc_alloc_fn alloc,
                                       bltc_free_fn free_fn, void* user);
/* Waits for the context's stream.  Errors: CUDA. */
bltc_status bltc_synchronize(bltc_context* ctx);
/* The message of the last failed call on ctx ("" if none); valid until the next call. */
const char* bltc_last_error(const bltc_context* ctx);
int bltc_version(void);
/* Multiprocessor count of the context's device (the persistent sweep's grid unit). */
int bltc_device_sm_count(const bltc_context* ctx);
/* Number of CUDA kernels this context has launched so far (a diagnostic counter). */
int64_t bltc_context_launch_count(const bltc_context* ctx);
/* Enables (1) or disables (0) phase timing: CUDA events recorded on the context's stream
 * at the phase boundaries of bltc_solve / bltc_evaluate.  Errors: ARG, CUDA. */
bltc_status bltc_context_set_timing(bltc_context* ctx, int enable);
/* Milliseconds of the last timed bltc_solve (or bltc_evaluate), ms[7] = {trees, lists,
 * modified charges, work plan, sweep kernel, finalize, total}; -1 for a phase that was not
 * recorded.  Waits for the last recorded event.  Errors: ARG, CUDA. */
bltc_status bltc_last_timings(bltc_context* ctx, float* ms);

/* ---- A0: tree of source clusters / target batches (Sec. II-D, Sec. III-A) ---------- */

/* Builds the tree over the n particles (x, y, z, and charges q, or q = NULL for a target
 * tree), splitting every node holding more than max_leaf particles by the rules above.
 * The tree keeps its own permuted FP64 copy of the particles.  Synchronizes once per tree
 * level.  Errors: ARG (n < 1, n >= 2^31, max_leaf < 1, NULL pointer, non-finite
 * coordinate or charge), OOM, CUDA. */
bltc_status bltc_tree_build(bltc_context* ctx, const double* x, const double* y,
                            const double* z, const double* q, int64_t n, int32_t max_leaf,
                            bltc_tree** out);
void bltc_tree_destroy(bltc_tree* tree);
/* Sizes of a built tree: particles, nodes, leaves, levels (root only = 1).  Host out
 * pointers, each may be NULL. */
bltc_status bltc_tree_info(const bltc_tree* tree, int64_t* n_particles, int64_t* n_nodes,
                           int64_t* n_leaves, int32_t* n_levels);
/* Copies the tree to HOST arrays (each may be NULL), nodes in DFS pre-order:
 * perm[n] (original index of the i-th particle in tree order), begin/count[m],
 * parent[m] (-1 at the root), level[m], n_children[m], children[8*m] (-1 padded, in
 * increasing octant order), lo/hi/center[3*m] (x, y, z per node), radius[m].
 * Synchronizes.  Errors: ARG, CUDA. */
bltc_status bltc_tree_export(bltc_context* ctx, const bltc_tree* tree, int64_t* perm,
                             int64_t* begin, int64_t* count, int32_t* parent, int32_t* level,
                             int32_t* n_children, int32_t* children, double* lo, double* hi,
                             double* center, double* radius);

/* ---- A1: interaction lists (MAC of Eq. 13, ComputePotential of Algorithm 1) -------- */

/* For every target batch (leaf of `batches`, DFS order) walks Algorithm 1's
 * ComputePotential from the root of `sources` and records the clusters approximated
 * (MAC passes) and summed directly (leaf with a failed geometric test, or a cluster with
 * (n+1)^3 >= N_C), each list in the recursion's visit order.  Uses params->theta and
 * params->degree.  batches may equal sources.  Synchronizes.  Errors: ARG, OOM, CUDA. */
bltc_status bltc_lists_build(bltc_context* ctx, const bltc_tree* batches,
                             const bltc_tree* sources, const bltc_params* params,
                             bltc_lists** out);
/* The lists of some target batches only, for evaluating a sample of the targets (the
 * error of Eq. 16 on a subset of targets, Sec. IV).  `batches` is a HOST array of
 * n_batches batch indices (leaves of the batch tree in DFS order), strictly increasing;
 * every other batch gets empty lists, so bltc_evaluate with the result writes phi = 0
 * for its targets.  The result refers to the same trees as `lists` and is freed with
 * bltc_lists_destroy.  Synchronizes.  Errors: ARG (NULL, index out of range, not
 * increasing), OOM, CUDA. */
bltc_status bltc_lists_select(bltc_context* ctx, const bltc_lists* lists, const int32_t* batches,
                              int64_t n_batches, bltc_lists** out);
void bltc_lists_destroy(bltc_lists* lists);
bltc_status bltc_lists_info(const bltc_lists* lists, int64_t* n_batches, int64_t* n_approx,
                            int64_t* n_direct);
/* Copies the lists to HOST CSR arrays (each may be NULL): approx_off/direct_off
 * [n_batches+1] and approx_ids[n_approx]/direct_ids[n_direct] (source node ids, DFS
 * pre-order numbering).  Synchronizes.  Errors: ARG, CUDA. */
bltc_status bltc_lists_export(bltc_context* ctx, const bltc_lists* lists, int64_t* approx_off,
                              int64_t* approx_ids, int64_t* direct_off, int64_t* direct_ids);
/* Evaluated kernel interactions of one evaluation: sum over batches of N_B * N_C for the
 * direct list and N_B * (n+1)^3 for the approximation list.  Synchronizes. */
bltc_status bltc_stats(bltc_context* ctx, const bltc_lists* lists,
                       int64_t* n_direct_interactions, int64_t* n_approx_interactions);
/* Kernel evaluations bltc_evaluate performs for these lists with params->degree and
 * params->precision: the N_B * (n+1)^3 approximation terms plus the direct terms, where in
 * MIXED precision with batches = sources a leaf pair that is in each other's direct list
 * (a mutual pair) is evaluated once for both of its batches (Eq. 1 is symmetric in i, j for
 * the Coulomb and Yukawa kernels).  Not in the paper.  Builds the work plan if needed.
 * Synchronizes.  Errors: ARG, CUDA. */
bltc_status bltc_evaluations(bltc_context* ctx, bltc_lists* lists, const bltc_params* params,
                             int64_t* n_evaluations);

/* ---- A2: modified charges (Eq. 12; Eq. 14-15; exact hits, Sec. II-C) --------------- */

/* Computes qhat_k = sum_{y_j in C} L_k1(y_j1) L_k2(y_j2) L_k3(y_j3) q_j for every cluster
 * C of `sources` with more than (n+1)^3 particles that appears in an approximation list of
 * `lists` (every such cluster if lists is NULL).  The source tree must carry charges.
 * Stored in the tree for params->degree and params->precision.  Errors: ARG, STATE, OOM,
 * CUDA. */
bltc_status bltc_modified_charges(bltc_context* ctx, bltc_tree* sources,
                                  const bltc_lists* lists, const bltc_params* params);
/* Copies the modified charges to a HOST array qhat[n_nodes * (n+1)^3] (node in DFS order,
 * k = (k1*(n+1) + k2)*(n+1) + k3); clusters without modified charges get NaN.
 * Synchronizes.  Errors: ARG, STATE, CUDA. */
bltc_status bltc_modified_charges_export(bltc_context* ctx, const bltc_tree* sources,
                                         double* qhat);

/* ---- A3-A5: far-field and near-field sweeps and the per-target finalize ------------ */

/* phi[i] = sum over the approximation list of batch(i) of Eq. 11 plus sum over its direct
 * list of Eq. 9, for every target i of `batches`, written to the caller's device buffer
 * phi[n_targets] in the caller's original target order.  Needs bltc_modified_charges for
 * the same degree and precision.  Runs the far/near sweep as one persistent launch over a
 * work queue of (batch, list range) items, then sums each target's per-item partials in a
 * fixed order (deterministic).  In MIXED precision with batches == sources, a leaf pair in
 * each other's direct list is evaluated once for both batches (G is symmetric); see
 * bltc_evaluations.  Errors: ARG, STATE, OOM, CUDA. */
bltc_status bltc_evaluate(bltc_context* ctx, const bltc_lists* lists, const bltc_tree* batches,
                          const bltc_tree* sources, const bltc_params* params, double* phi);

/* The whole of Algorithm 1 with targets = sources: builds the source tree (leaf_size) and
 * the batch tree (batch_size; shared when equal), the lists, the modified charges, and
 * evaluates phi[n] (device, original order).  Errors: as the steps above. */
bltc_status bltc_solve(bltc_context* ctx, const double* x, const double* y, const double* z,
                       const double* q, int64_t n, const bltc_params* params, double* phi);

/* Algorithm 1 for distinct target and source sets (Sec. II: the treecode needs only target
 * and source positions; the paper's runs use targets = sources).  nt targets (tx, ty, tz),
 * ns sources (sx, sy, sz) with charges sq, all DEVICE pointers owned by the caller.  Builds
 * the source tree with params->leaf_size (N_L) and the batch tree of the targets with
 * params->batch_size (N_B), then lists, modified charges and the sweeps; phi[nt] (device)
 * receives the potentials in the caller's target order.  A target at exactly the position of
 * a source skips that pair (r^2 == 0), as in bltc_solve.  Errors: as bltc_solve. */
bltc_status bltc_solve_targets(bltc_context* ctx, const double* tx, const double* ty,
                               const double* tz, int64_t nt, const double* sx, const double* sy,
                               const double* sz, const double* sq, int64_t ns,
                               const bltc_params* params, double* phi);

/* The cluster-particle variant (the paper's future work, Sec. V): the roles of Algorithm 1
 * swapped.  Targets (tx, ty, tz; nt) form the clusters, in a tree with params->leaf_size,
 * and are interpolated; sources (sx, sy, sz, sq; ns) form the batches, leaves of a tree with
 * params->batch_size, and are summed exactly.  For every source batch S, ComputePotential
 * walks the target tree with the MAC of Eq. 13 ((r_S + r_T)/R < theta and (n+1)^3 < N_T):
 * an approximated target cluster T accumulates phihat_T[k] = sum_{y_j in S} G(t_k, y_j) q_j
 * at its Chebyshev points t_k; a direct one adds sum_{y_j in S} G(x_i, y_j) q_j to each of
 * its targets.  Finally phi(x_i) += sum_k L_k1 L_k2 L_k3 (x_i) phihat_T[k] (Eq. 4-8, exact
 * hits) for every cluster T holding x_i.  Device pointers; phi[nt] in the caller's target
 * order.  Built-in and registered kernels, both precisions (the interpolation runs in FP64).
 * Errors: as bltc_solve. */
bltc_status bltc_solve_cp(bltc_context* ctx, const double* tx, const double* ty, const double* tz,
                          int64_t nt, const double* sx, const double* sy, const double* sz,
                          const double* sq, int64_t ns, const bltc_params* params, double* phi);

/* The cluster-cluster variant (dual tree traversal; the paper's future work, Sec. V).
 * Sources (sx, sy, sz, sq; ns) in a tree with params->leaf_size, targets (tx, ty, tz; nt) in
 * a tree with params->batch_size.  DualTraversal(T, S) from the two roots: if
 * (r_T + r_S)/R < theta (Eq. 13) the pair interacts as CC when (n+1)^3 < N_T and
 * (n+1)^3 < N_S (point potentials of T's Chebyshev grid from S's modified charges), CP when
 * only (n+1)^3 < N_T (from S's particles), PC when only (n+1)^3 < N_S (T's targets from S's
 * modified charges), PP otherwise (exact); else leaf-leaf pairs are PP and otherwise T is
 * split when S is a leaf or (T is not a leaf and r_T >= r_S), S otherwise, children in stored
 * order.  Each target then adds the interpolants (Eq. 4-8, exact hits) of its clusters'
 * point potentials.  Device pointers; phi[nt] in the caller's target order.  Errors: as
 * bltc_solve. */
bltc_status bltc_solve_cc(bltc_context* ctx, const double* tx, const double* ty, const double* tz,
                          int64_t nt, const double* sx, const double* sy, const double* sz,
                          const double* sq, int64_t ns, const bltc_params* params, double* phi);
/* The dual traversal's interaction lists for two trees (params->theta, params->degree):
 * counts[4] = the numbers of CC, CP, PC and PP pairs; target_ids / source_ids (HOST arrays of
 * sum(counts), or NULL for the counts only) receive the pairs' node ids (DFS pre-order),
 * the four lists one after the other, each level by level in traversal order.  Synchronizes.
 * Errors: ARG, OOM, CUDA. */
bltc_status bltc_dual_lists(bltc_context* ctx, const bltc_tree* targets, const bltc_tree* sources,
                            const bltc_params* params, int64_t* counts, int64_t* target_ids,
                            int64_t* source_ids);

/* The barycentric Hermite treecode (the paper's future work, Sec. V), targets =
 * sources.  On the n+1 Chebyshev points of each approximated cluster the kernel is
 * interpolated with values and first derivatives (H_k = (1 - 2 L_k'(s_k)(y - s_k)) L_k^2,
 * K_k = (y - s_k) L_k^2; exact hits give H = e_m, K = 0), exact for degree 2n+1:
 * phi(x_i) ~ sum_k sum_a D^a G(x_i, s_k) qhat^a_k over the 8 mixed derivatives
 * a in {0,1}^3, with qhat^a_k = sum_j q_j B^a1_k1 B^a2_k2 B^a3_k3 (y_j), B^0 = H, B^1 = K.
 * The MAC is Eq. 13 with the size test 8 (n+1)^3 < N_C.  params->precision FP64, or MIXED
 * (the far field's 8 terms in FP32 on batch-relative coordinates with FP32 charges, the
 * treecode's mixed near field, FP64 accumulation); 1 <= params->degree <= 7, kernel Coulomb or
 * Yukawa.  Device pointers, phi[n] in the caller's order.  Errors: as bltc_solve (ARG for the
 * restrictions above). */
bltc_status bltc_solve_hermite(bltc_context* ctx, const double* x, const double* y, const double* z,
                               const double* q, int64_t n, const bltc_params* params, double* phi);

/* A solve with fixed positions, replayed as one CUDA graph (Algorithm 1 with its setup done
 * once).  Trees (Sec. II-D), lists (Eq. 13) and the work plans depend only on the positions;
 * the upward pass (Eq. 12) and the sweep (Eq. 9, 11) depend on the charges.  Iterative methods
 * that apply the same interaction to a new charge vector at every step replay only the latter.
 *
 * bltc_graph_create builds the trees and lists for x, y, z (device, n particles, targets =
 * sources), runs one solve with the charges q into phi (as bltc_solve), allocates every buffer a
 * replay needs and captures on a private stream: the gather of q into tree order, the upward
 * pass, the sweep and the finalize into phi.  q and phi (device, n, caller order) are BOUND: each
 * bltc_graph_launch reads the charges currently in q and overwrites phi, as one cudaGraphLaunch on
 * the context's stream, with no host synchronisation and no allocation.  The positions are copied
 * at creation; later changes to x, y, z are not seen.  Parameters as bltc_solve (built-in or
 * registered kernels, FP64 or mixed); results of a launch are the bits bltc_solve gives for the
 * same positions and charges.  The graph holds device memory of the context and must be destroyed
 * before it; q and phi must stay allocated while the graph is launched.
 * Errors: ARG (parameters, NULL pointers), OOM, CUDA; STATE if launched on another context.
 * bltc_graph_kernels returns the kernels one launch runs (-1 for NULL). */
bltc_status bltc_graph_create(bltc_context* ctx, const double* x, const double* y, const double* z,
                              const double* q, int64_t n, const bltc_params* params, double* phi,
                              bltc_graph** out);
bltc_status bltc_graph_launch(bltc_context* ctx, bltc_graph* graph);
int64_t bltc_graph_kernels(const bltc_graph* graph);
void bltc_graph_destroy(bltc_graph* graph);

/* A solve for NEW positions at every launch, as one CUDA graph: the whole of Algorithm 1
 * (tree and batches, Sec. II-D; lists, Eq. 13; modified charges, Eq. 12; far and near field,
 * Eq. 11 and 9; the fixed-order finalize), with no host synchronisation between the tree and
 * the finalize.  The host-driven bltc_solve reads counts back at every step to size the next;
 * here every buffer has a capacity and every count stays in device memory.
 *
 * bltc_graph_create_positions solves once with x, y, z, q into phi (as bltc_solve), sets the
 * capacities to that solve's counts (tree nodes and levels, list entries, clusters with
 * modified charges, work items, partial and mutual-row lengths) times `headroom` (0 selects
 * 1.25; else 1 <= headroom <= 16) plus a margin, and captures the sized solve.  x, y, z, q and
 * phi (device, n, caller order) are BOUND: each bltc_graph_launch reads the positions and
 * charges currently in them and overwrites phi.  A launch is one cudaGraphLaunch followed by a
 * read of a 4-byte flag, so it SYNCHRONIZES.  Results are the bits bltc_solve gives for the same
 * inputs.  If the positions need more than a capacity (or are not finite), the sized solve raises
 * the flag without writing past any buffer; the launch then solves again on the host-driven path
 * (which reports non-finite input as ARG) and rebuilds the graph for the new sizes, so phi is
 * always correct.  Parameters as bltc_solve (built-in or registered kernels, FP64 or mixed, leaf
 * and batch sizes may differ).  Memory: the graph holds every buffer of one solve at its capacity
 * (about the footprint of a bltc_solve times the headroom).  Errors: as bltc_graph_create.
 *
 * bltc_graph_info writes {kernels per launch, launches, launches redone on the host path,
 * captures} of either kind of graph to out[4]; ARG for NULL. */
bltc_status bltc_graph_create_positions(bltc_context* ctx, const double* x, const double* y,
                                        const double* z, const double* q, int64_t n,
                                        const bltc_params* params, double* phi, double headroom,
                                        bltc_graph** out);
bltc_status bltc_graph_info(const bltc_graph* graph, int64_t* out);

/* bltc_solve for HOST buffers x, y, z, q, phi (pinned memory recommended): copies the
 * inputs to the device, solves, copies phi back.  Synchronizes.  Errors: as bltc_solve. */
bltc_status bltc_solve_host(bltc_context* ctx, const double* x, const double* y,
                            const double* z, const double* q, int64_t n,
                            const bltc_params* params, double* phi);

/* ---- autotuning of the leaf and batch sizes --------------------------------------- */

/* Chooses the leaf and batch sizes of the given system among candidate pairs (leaf[i],
 * batch[i]; batch may be NULL for batch = leaf).  Not in the paper.  First a screen: the
 * trees, lists and sweep plan of every candidate give its exact work in padded target slots
 * (each batch's targets rounded up to the passes of its source groups, times the sources
 * and proxy points it meets); candidates with the same trees count once.  Then the
 * contenders, at most 3 distinct candidates within 10% of the smallest work, are timed with
 * bltc_solve (one warm-up, then `repeats` runs, the fastest counts) and the fastest wins;
 * a single contender wins untimed.  Writes the choice into *best (a copy of *params with
 * those sizes) and every candidate's fastest time into ms[n_candidates] (may be NULL; NaN
 * for a candidate not timed).  The choice is cached in the context under (floor(log2 n),
 * degree, kernel, precision, theta to 1e-3, mean batch size of the first candidate in
 * quarter octaves): a later call with the same key and use_cache != 0 returns it untimed,
 * after screening the first candidate only, if it is among that call's candidates.  Device pointers as bltc_solve.  Synchronizes.  Errors: ARG, OOM, CUDA. */
bltc_status bltc_autotune(bltc_context* ctx, const double* x, const double* y, const double* z,
                          const double* q, int64_t n, const bltc_params* params,
                          const int32_t* leaf, const int32_t* batch, int32_t n_candidates,
                          int32_t repeats, int32_t use_cache, bltc_params* best, float* ms);

/* Chooses the mixed sweep's tile shape (params->tile) for the given system at the leaf and
 * batch sizes of *params, among candidates tiles[n_tiles] (0 included for the defaults).  Not
 * in the paper.  Each candidate is timed with bltc_solve (one warm-up, then `repeats` runs, the
 * fastest counts); the fastest wins.  Writes *params with that tile into *best and every
 * candidate's time into ms[n_tiles] (may be NULL).  Cached in the context under
 * (floor(log2 n), degree, kernel, precision, theta to 1e-3, mean batch size in quarter
 * octaves, leaf and batch size): a later call with that key and use_cache != 0 returns the
 * choice untimed if it is among its candidates.  Device pointers as bltc_solve.  Synchronizes.
 * Errors: ARG (a malformed tile, no candidates), OOM, CUDA. */
bltc_status bltc_autotune_tile(bltc_context* ctx, const double* x, const double* y, const double* z,
                               const double* q, int64_t n, const bltc_params* params,
                               const int32_t* tiles, int32_t n_tiles, int32_t repeats,
                               int32_t use_cache, bltc_params* best, float* ms);

/* ---- user kernels: a hook for any smooth, non-oscillatory radial G ---------------- */
/* The treecode needs only evaluations of G (Sec. I; Sec. V names other kernels as the
 * method's generality).  `source` is CUDA C++ source that defines
 *     __device__ float  bltc_user_g32(float r2, float r, float param);
 *     __device__ double bltc_user_g64(double r2, double r, double param);
 * returning G at distance r = sqrt(r2) > 0 in FP32 (MIXED) and FP64; param is
 * params->kappa.  G must depend on r only (the mixed sweep evaluates a mutual leaf pair once
 * for both of its batches).  Pairs with r^2 == 0 are skipped as for the built-in kernels.
 * The library compiles its sweep kernels with these functions at run time with NVRTC
 * (libnvrtc.so of the CUDA toolkit, loaded on first use; BLTC_NVRTC_PATH may name it) for
 * the context's device, and writes the id to use as params->kernel in this context:
 * bltc_solve, bltc_solve_targets, bltc_evaluate and bltc_autotune accept it; the direct sum
 * and the serving runtime take the built-in kernels only.
 * Errors: ARG (NULL arguments, or the source does not compile: the compiler log is in
 * bltc_last_error), STATE (NVRTC not found), CUDA. */
bltc_status bltc_kernel_register(bltc_context* ctx, const char* source, int32_t* kernel_id);
/* Compiles a user kernel source for sm_<arch> (e.g. 103) without a device, as a check.
 * Copies the compiler log to log[len] (may be NULL) and returns BLTC_OK if it compiled, ARG
 * if not, STATE if NVRTC is not found. */
bltc_status bltc_kernel_check(const char* source, int32_t arch, char* log, int64_t len);

/* ---- direct summation, Eq. 1 (the GPU baseline) ----------------------------------- */

/* phi[i] = sum_j G(x_i, y_j) q_j over all nt targets (tx, ty, tz) and ns sources
 * (sx, sy, sz, sq), pairs with r^2 == 0 skipped; params->kernel, kappa and precision are
 * used (MIXED: FP32 evaluation on absolute coordinates, FP32 sums over tiles of sources,
 * FP64 across tiles).  Device pointers.  Errors: ARG, OOM, CUDA. */
bltc_status bltc_direct_sum(bltc_context* ctx, const double* tx, const double* ty,
                            const double* tz, int64_t nt, const double* sx, const double* sy,
                            const double* sz, const double* sq, int64_t ns,
                            const bltc_params* params, double* phi);

/* bltc_direct_sum for callers that cannot allocate device memory: applications whose device
 * heap belongs to another allocator (a host framework's pool, a fixed arena) and that may
 * not call cudaMalloc or free memory behind it.  This entry point allocates nothing: the
 * per-split partial sums go to a fixed scratch array of 64 MiB (8,388,608 doubles) compiled
 * into the library, which every GPU that loads the library holds until the process exits.
 * No counterpart in the paper.
 *   - Same arguments, results and tolerances as bltc_direct_sum; the caller still passes
 *     the inputs and phi.  nt must be at most 8,388,608 (else BLTC_ERR_ARG); the number of
 *     source splits is limited so that splits * nt partial sums fit the scratch.
 *   - The first call on a device looks up the scratch's device address once (with that
 *     device current); make that first call before any stream capture.
 *   - Every call on a device shares the one scratch array: calls that overlap on the GPU
 *     (two streams, or two contexts at once) race and corrupt each other's sums; serialise
 *     them.  The array keeps the last call's contents; every partial sum a call reads is
 *     written by that same call, so nothing needs clearing.
 * Errors: ARG, CUDA. */
bltc_status bltc_direct_sum_noalloc(bltc_context* ctx, const double* tx, const double* ty,
                                    const double* tz, int64_t nt, const double* sx,
                                    const double* sy, const double* sz, const double* sq,
                                    int64_t ns, const bltc_params* params, double* phi);

/* ---- serving: continuous batching of many requests on one GPU -------------------- */
/* Not in the paper (which runs one system per rank); the runtime that keeps the GPU busy
 * with a stream of independent particle systems of uneven size.  Each request is the whole
 * of Algorithm 1 in mixed precision (targets = sources).  Requests are admitted in
 * arrival order while their estimated device memory fits the HBM budget; setup workers
 * (host threads with their own streams) build each admitted request's tree, lists,
 * modified charges and work plan; one engine merges the far/near sweeps of the prepared
 * requests into persistent launches (work items of all their requests, longest first), in
 * slices of about slice_us microseconds that favour the requests with the least remaining
 * work, then finalizes each request and copies its potentials out.  Setup of later requests overlaps
 * the running sweep.  A request's potentials are bit-identical to bltc_solve of that
 * request alone, whatever else is in flight. */

typedef struct bltc_server bltc_server;

typedef struct bltc_server_config {
    int32_t device;           /* CUDA device */
    int32_t setup_workers;    /* host threads preparing requests, 1..64 */
    int32_t max_batch;        /* most requests one slice takes work from, >= 1 */
    int32_t linger_us;        /* batching window, >= 0: with fewer than max_batch requests
                               * ready while others are still being prepared, the engine
                               * waits up to this many microseconds for them before it
                               * launches (0: launch at once) */
    int64_t hbm_budget_bytes; /* device bytes admitted requests may reserve; 0 = 80% of free */
    int32_t slice_us;         /* >= 0: the engine runs the ready work in slices of about this
                               * many microseconds of device time (converted to work by the
                               * rate its earlier launches ran at), the requests with the least
                               * remaining work first, so a request that arrives during a large
                               * sweep starts at the next slice; 0: all ready work in one slice */
    int32_t setup_blocks;     /* >= 0: block slots (of 2 per SM) the slices' sweeps leave free
                               * for the kernels of requests in preparation, which otherwise
                               * wait for a slice to end; setup workers' streams also take the
                               * device's greatest stream priority (0: the sweeps fill every
                               * slot) */
    int32_t slices_in_flight; /* 0, 1 or 2: slices enqueued on the device at a time (0: 1).  The
                               * engine takes the requests that became ready just before it
                               * assembles a slice, after the slice before has run (1) or while
                               * it runs (2): with 1 a new request waits about one slice less,
                               * at the cost of the host time between slices.  Slices are sized
                               * by the rate the engine's launches have measured */
} bltc_server_config;

typedef struct bltc_request_info {
    int32_t status;           /* bltc_status of the request */
    int32_t batch;            /* requests in the last slice it ran in */
    int64_t bytes_reserved;   /* device bytes reserved for it at admission */
    double t_submit, t_admit, t_ready, t_done;   /* host monotonic clock, seconds */
    double t_swept;           /* when the engine enqueued its last items and its finalize */
    double t_copy;            /* when its finalize had completed and the copy-out began */
} bltc_request_info;

typedef struct bltc_server_stats {
    int64_t submitted, completed, failed, cancelled, queued;
    int64_t sweep_launches, max_batch;
    int64_t budget_bytes, reserved_bytes, peak_reserved_bytes;
    int64_t live_bytes, peak_live_bytes;   /* actually allocated through the server */
} bltc_server_counters;

/* Starts the server threads on cfg->device.  Errors: ARG, CUDA. */
bltc_status bltc_server_create(const bltc_server_config* cfg, bltc_server** out);
/* Queues one request.  x, y, z, q (inputs) and phi (output, n values in input order) are
 * HOST pointers that the caller keeps valid until bltc_server_wait has returned for the
 * ticket (pinned memory is faster).  params->precision must be BLTC_PRECISION_MIXED.
 * Returns at once with *ticket.  Errors: ARG (bad sizes or parameters), OOM (the request
 * alone exceeds the budget), STATE (server shutting down). */
bltc_status bltc_server_submit(bltc_server* server, const double* x, const double* y,
                               const double* z, const double* q, int64_t n,
                               const bltc_params* params, double* phi, uint64_t* ticket);
/* Waits for a request (timeout_s < 0: no limit), fills *info (may be NULL) and retires the
 * ticket.  Returns the request's status; TIMEOUT if it is still running (the ticket stays
 * valid); ARG for an unknown ticket. */
bltc_status bltc_server_wait(bltc_server* server, uint64_t ticket, double timeout_s,
                             bltc_request_info* info);
/* Cancels a request that has not been admitted (its wait returns CANCELLED).  Errors: ARG
 * (unknown ticket), STATE (already admitted). */
bltc_status bltc_server_cancel(bltc_server* server, uint64_t ticket);
bltc_status bltc_server_stats(bltc_server* server, bltc_server_counters* out);
/* Copies the message of the most recently failed request (empty if none) into buf (len
 * bytes, NUL-terminated, truncated to fit; buf may be NULL) and returns its full length, or
 * -1 for a NULL server. */
int64_t bltc_server_last_error(bltc_server* server, char* buf, int64_t len);
/* Cancels queued requests, lets admitted ones finish, stops the threads. */
void bltc_server_destroy(bltc_server* server);

#ifdef __cplusplus
}
#endif
#endif /* BLTC_H */
