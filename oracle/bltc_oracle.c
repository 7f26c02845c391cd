/*
 * bltc_oracle.c -- plain FP64 CPU oracle of the barycentric Lagrange treecode (BLTC)
 * of Vaughn, Wilson and Krasny, "A GPU-Accelerated Barycentric Lagrange Treecode".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct reference that the
 * CUDA library is checked against.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline and reference legs may load it.  It shares no code, header, table or helper with the
 * library; both receive the same input arrays from the seeded generators and nothing else.
 *
 * Everything is IEEE FP64, compiled with -ffp-contract=off so that a*b+c is never fused.
 * OpenMP is used only across independent units (targets of the direct sum, clusters of the
 * upward pass, target batches of the treecode), as the paper's CPU code did (Sec. IV,
 * "Single GPU vs. Single 6-Core CPU").  The order of every floating-point sum is fixed.
 *
 * Readings of the paper taken where it is silent (each is restated where it is used):
 *   R1  a pair with r^2 == 0 exactly is skipped (targets equal sources, Eq. 1);
 *   R2  cluster and batch boxes are the minimal axis-aligned boxes of their particles;
 *       min/max order -0.0 before +0.0;
 *   R3  centre c = 0.5*(lo+hi), half extent h = 0.5*(hi-lo), radius sqrt(hx*hx+hy*hy+hz*hz),
 *       R = sqrt(dx*dx+dy*dy+dz*dz) between centres, all left to right;
 *   R4  the geometric MAC test is (rB+rC)/R < theta (IEEE division); a NaN ratio fails it;
 *   R5  Algorithm 1's branch order, a size-rejected cluster is summed directly whole;
 *   R6  split rule: dimension d is split iff (hi_d-lo_d)*sqrt(2) >= max extent; a particle
 *       goes low iff coord < 0.5*(lo_d+hi_d); octant bit0/1/2 = x/y/z high; children in
 *       increasing octant order, empty ones dropped; stable partition; leaf iff count <=
 *       max_leaf, or zero extent, or the split leaves one non-empty child; DFS pre-order ids;
 *   R7  Chebyshev points s_k = lo + 0.5*(t_k+1)*(hi-lo), t_k = cos(pi*k/n), with s_0 = hi
 *       and s_n = lo forced;
 *   R8  exact hit in dimension l iff |y - s_k| < DBL_MIN, smallest such k wins.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "bltc_oracle.h"

/* ------------------------------------------------------------------------------------ */
/* Kernels G(x, y), Eq. 2, plus a polynomial test kernel.                                 */
/* ------------------------------------------------------------------------------------ */

/* Polynomial test kernel (not in the paper): G(x, y) = prod_l (1 + x_l*y_l/2)^n.  Its degree
 * in every source coordinate y_l is n, so the tensor-product interpolant of Eq. 8 reproduces
 * it exactly and the treecode must equal the direct sum up to rounding. */
static double poly_kernel(int degree, double tx, double ty, double tz,
                          double sx, double sy, double sz)
{
    double fx = 1.0 + 0.5 * tx * sx;
    double fy = 1.0 + 0.5 * ty * sy;
    double fz = 1.0 + 0.5 * tz * sz;
    double g = 1.0;
    for (int m = 0; m < degree; ++m) g = g * fx;
    for (int m = 0; m < degree; ++m) g = g * fy;
    for (int m = 0; m < degree; ++m) g = g * fz;
    return g;
}

/* G(x_i, y_j) of Eq. 2.  Returns 0 (pair skipped, reading R1) when r^2 == 0, else 1. */
static int kernel_G(int kernel, double kappa, int degree,
                    double tx, double ty, double tz, double sx, double sy, double sz,
                    double* g)
{
    double dx = tx - sx;
    double dy = ty - sy;
    double dz = tz - sz;
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return 0;
    if (kernel == ORACLE_KERNEL_POLY) {
        *g = poly_kernel(degree, tx, ty, tz, sx, sy, sz);
        return 1;
    }
    if (kernel == ORACLE_KERNEL_SOFT) {
        /* softened Coulomb 1/sqrt(r^2 + eps^2), eps = kappa: a smooth, non-oscillatory
         * radial kernel outside Eq. 2, as the method allows (Sec. I, Sec. V) */
        *g = 1.0 / sqrt(r2 + kappa * kappa);
        return 1;
    }
    double r = sqrt(r2);
    if (kernel == ORACLE_KERNEL_YUKAWA)
        *g = exp(-kappa * r) / r;       /* Yukawa, Eq. 2 right */
    else
        *g = 1.0 / r;                   /* Coulomb, Eq. 2 left */
    return 1;
}

/* ------------------------------------------------------------------------------------ */
/* Direct summation, Eq. 1.                                                              */
/* ------------------------------------------------------------------------------------ */

int oracle_direct_sum(const double* tx, const double* ty, const double* tz, int64_t nt,
                      const double* sx, const double* sy, const double* sz, const double* sq,
                      int64_t ns, int32_t kernel, double kappa, int32_t degree,
                      int32_t threads, double* phi, double* phi_abs)
{
    if (nt < 0 || ns < 0) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
    /* phi(x_i) = sum_j G(x_i, y_j) q_j, j ascending. */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nt; ++i) {
        double acc = 0.0, acc_abs = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            double g;
            if (!kernel_G(kernel, kappa, degree, tx[i], ty[i], tz[i], sx[j], sy[j], sz[j], &g))
                continue;
            acc = acc + g * sq[j];
            acc_abs = acc_abs + fabs(g * sq[j]);
        }
        phi[i] = acc;
        if (phi_abs) phi_abs[i] = acc_abs;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Tree of source clusters / target batches, Sec. II-D "Source Clusters and Target        */
/* Batches" and the aspect-ratio rule of Sec. III-A (readings R2, R3, R6).                */
/* ------------------------------------------------------------------------------------ */

struct oracle_tree {
    int64_t n;            /* particles */
    int64_t n_nodes, cap;
    int64_t* perm;        /* perm[i] = original index of the i-th particle in tree order */
    int64_t* begin;       /* node's first position in tree order */
    int64_t* count;       /* node's particle count */
    int32_t* parent;      /* -1 for the root */
    int32_t* level;       /* root = 0 */
    int32_t* n_children;  /* 0 for a leaf */
    int32_t* children;    /* 8 per node, in increasing octant order, -1 padded */
    double* lo;           /* 3 per node: minimal box */
    double* hi;
    double* center;       /* 3 per node */
    double* radius;
};

static int tree_grow(oracle_tree* t)
{
    if (t->n_nodes < t->cap) return 0;
    int64_t cap = t->cap ? 2 * t->cap : 64;
#define GROW(field, type, per)                                                      \
    do {                                                                            \
        type* p = (type*)realloc(t->field, (size_t)(cap * (per)) * sizeof(type));   \
        if (!p) return -1;                                                          \
        t->field = p;                                                               \
    } while (0)
    GROW(begin, int64_t, 1);
    GROW(count, int64_t, 1);
    GROW(parent, int32_t, 1);
    GROW(level, int32_t, 1);
    GROW(n_children, int32_t, 1);
    GROW(children, int32_t, 8);
    GROW(lo, double, 3);
    GROW(hi, double, 3);
    GROW(center, double, 3);
    GROW(radius, double, 1);
#undef GROW
    t->cap = cap;
    return 0;
}

/* Total order on the box coordinates: -0.0 sorts before +0.0 (reading R2). */
static int less_total(double a, double b)
{
    return a < b || (a == b && signbit(a) && !signbit(b));
}

typedef struct {
    const double* c[3];   /* x, y, z in original order */
    int32_t max_leaf;
    uint8_t* oct;         /* scratch: octant code per tree position */
    int64_t* tmp;         /* scratch: partition buffer */
} build_ctx;

/* Builds the node covering tree positions [begin, begin+count) and its subtree.
 * Returns the node id (DFS pre-order), or -1 on allocation failure. */
static int64_t build_node(oracle_tree* t, build_ctx* b, int64_t begin, int64_t count,
                          int32_t parent, int32_t level)
{
    if (tree_grow(t)) return -1;
    int64_t id = t->n_nodes++;
    t->begin[id] = begin;
    t->count[id] = count;
    t->parent[id] = parent;
    t->level[id] = level;
    t->n_children[id] = 0;
    for (int c = 0; c < 8; ++c) t->children[8 * id + c] = -1;

    /* Minimal bounding box of the node's own particles (R2). */
    double lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        lo[d] = b->c[d][t->perm[begin]];
        hi[d] = lo[d];
        for (int64_t i = begin + 1; i < begin + count; ++i) {
            double v = b->c[d][t->perm[i]];
            if (less_total(v, lo[d])) lo[d] = v;
            if (less_total(hi[d], v)) hi[d] = v;
        }
    }
    /* Centre and radius (R3). */
    double h[3];
    for (int d = 0; d < 3; ++d) {
        t->lo[3 * id + d] = lo[d];
        t->hi[3 * id + d] = hi[d];
        t->center[3 * id + d] = 0.5 * (lo[d] + hi[d]);
        h[d] = 0.5 * (hi[d] - lo[d]);
    }
    t->radius[id] = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);

    /* Recursion stops at max_leaf particles or fewer (Sec. II-D). */
    if (count <= b->max_leaf) return id;
    double L[3], Lmax = 0.0;
    for (int d = 0; d < 3; ++d) {
        L[d] = hi[d] - lo[d];
        if (L[d] > Lmax) Lmax = L[d];
    }
    if (Lmax == 0.0) return id;

    /* Aspect-ratio rule (Sec. III-A): split only the dimensions whose extent is within a
     * factor sqrt(2) of the longest; the longest always splits. */
    int split[3];
    double mid[3];
    for (int d = 0; d < 3; ++d) {
        split[d] = (L[d] * 1.4142135623730951 >= Lmax);
        mid[d] = 0.5 * (lo[d] + hi[d]);
    }

    /* Octant of each particle: bit d set iff dimension d is split and coord >= midpoint. */
    int64_t cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = begin; i < begin + count; ++i) {
        int o = 0;
        for (int d = 0; d < 3; ++d)
            if (split[d] && !(b->c[d][t->perm[i]] < mid[d])) o |= (1 << d);
        b->oct[i] = (uint8_t)o;
        cnt[o]++;
    }
    int nonempty = 0;
    for (int o = 0; o < 8; ++o) nonempty += (cnt[o] > 0);
    if (nonempty <= 1) return id;   /* the split makes no progress: keep as a leaf (R6) */

    /* Stable partition of perm[begin, begin+count) by octant. */
    int64_t k = 0;
    for (int o = 0; o < 8; ++o)
        for (int64_t i = begin; i < begin + count; ++i)
            if (b->oct[i] == o) b->tmp[k++] = t->perm[i];
    memcpy(t->perm + begin, b->tmp, (size_t)count * sizeof(int64_t));

    /* Children in increasing octant order; ids are assigned on entry (DFS pre-order). */
    int64_t sub = begin;
    int nc = 0;
    for (int o = 0; o < 8; ++o) {
        if (cnt[o] == 0) continue;
        int64_t child = build_node(t, b, sub, cnt[o], (int32_t)id, level + 1);
        if (child < 0) return -1;
        t->children[8 * id + nc] = (int32_t)child;
        nc++;
        sub += cnt[o];
    }
    t->n_children[id] = nc;
    return id;
}

void oracle_tree_free(oracle_tree* t)
{
    if (!t) return;
    free(t->perm);
    free(t->begin);
    free(t->count);
    free(t->parent);
    free(t->level);
    free(t->n_children);
    free(t->children);
    free(t->lo);
    free(t->hi);
    free(t->center);
    free(t->radius);
    free(t);
}

int oracle_tree_build(const double* x, const double* y, const double* z, int64_t n,
                      int32_t max_leaf, oracle_tree** out)
{
    *out = NULL;
    if (n < 1 || max_leaf < 1) return -1;
    oracle_tree* t = (oracle_tree*)calloc(1, sizeof(oracle_tree));
    if (!t) return -2;
    t->n = n;
    t->perm = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    build_ctx b;
    b.c[0] = x;
    b.c[1] = y;
    b.c[2] = z;
    b.max_leaf = max_leaf;
    b.oct = (uint8_t*)malloc((size_t)n);
    b.tmp = (int64_t*)malloc((size_t)n * sizeof(int64_t));
    if (!t->perm || !b.oct || !b.tmp) {
        free(b.oct);
        free(b.tmp);
        oracle_tree_free(t);
        return -2;
    }
    for (int64_t i = 0; i < n; ++i) t->perm[i] = i;
    int64_t root = build_node(t, &b, 0, n, -1, 0);
    free(b.oct);
    free(b.tmp);
    if (root != 0) {
        oracle_tree_free(t);
        return -2;
    }
    *out = t;
    return 0;
}

int64_t oracle_tree_num_nodes(const oracle_tree* t) { return t->n_nodes; }

void oracle_tree_export(const oracle_tree* t, int64_t* perm, int64_t* begin, int64_t* count,
                        int32_t* parent, int32_t* level, int32_t* n_children,
                        int32_t* children, double* lo, double* hi, double* center,
                        double* radius)
{
    int64_t m = t->n_nodes;
    if (perm) memcpy(perm, t->perm, (size_t)t->n * sizeof(int64_t));
    if (begin) memcpy(begin, t->begin, (size_t)m * sizeof(int64_t));
    if (count) memcpy(count, t->count, (size_t)m * sizeof(int64_t));
    if (parent) memcpy(parent, t->parent, (size_t)m * sizeof(int32_t));
    if (level) memcpy(level, t->level, (size_t)m * sizeof(int32_t));
    if (n_children) memcpy(n_children, t->n_children, (size_t)m * sizeof(int32_t));
    if (children) memcpy(children, t->children, (size_t)(8 * m) * sizeof(int32_t));
    if (lo) memcpy(lo, t->lo, (size_t)(3 * m) * sizeof(double));
    if (hi) memcpy(hi, t->hi, (size_t)(3 * m) * sizeof(double));
    if (center) memcpy(center, t->center, (size_t)(3 * m) * sizeof(double));
    if (radius) memcpy(radius, t->radius, (size_t)m * sizeof(double));
}

/* ------------------------------------------------------------------------------------ */
/* Barycentric Lagrange interpolation, Sec. II-A and II-C.                               */
/* ------------------------------------------------------------------------------------ */

/* Chebyshev points of the second kind mapped to [lo, hi] (Eq. 6, reading R7) and their
 * barycentric weights (Eq. 7), which the linear map leaves unchanged. */
void oracle_cheb(int32_t degree, double lo, double hi, double* s, double* w)
{
    const double pi = 3.14159265358979323846;
    for (int k = 0; k <= degree; ++k) {
        double tk = cos(pi * (double)k / (double)degree);
        s[k] = lo + 0.5 * (tk + 1.0) * (hi - lo);
        double delta = (k == 0 || k == degree) ? 0.5 : 1.0;
        w[k] = ((k % 2) ? -1.0 : 1.0) * delta;
    }
    s[0] = hi;
    s[degree] = lo;
}

/* The n+1 values L_k(y), k = 0..n, of Eq. 4 on the Chebyshev points of [lo, hi].  When y
 * coincides with a point s_k' (|y - s_k'| below the smallest positive normal double,
 * Sec. II-C), L_k(y) = delta_{k k'} is enforced instead (reading R8: smallest k'). */
void oracle_lagrange(int32_t degree, double lo, double hi, double y, double* a)
{
    double s[ORACLE_MAX_DEGREE + 1], w[ORACLE_MAX_DEGREE + 1];
    oracle_cheb(degree, lo, hi, s, w);
    for (int k = 0; k <= degree; ++k) {
        if (fabs(y - s[k]) < DBL_MIN) {
            for (int m = 0; m <= degree; ++m) a[m] = (m == k) ? 1.0 : 0.0;
            return;
        }
    }
    double denom = 0.0;
    for (int k = 0; k <= degree; ++k) denom = denom + w[k] / (y - s[k]);
    for (int k = 0; k <= degree; ++k) a[k] = (w[k] / (y - s[k])) / denom;
}

/* Modified charges of every cluster, Eq. 12 (Algorithm 1, the loop over source clusters):
 * qhat_k = sum_{y_j in C} L_k1(y_j1) L_k2(y_j2) L_k3(y_j3) q_j, j in tree order,
 * k = (k1*(n+1) + k2)*(n+1) + k3.  qhat has n_nodes*(n+1)^3 entries. */
int oracle_modified_charges(const oracle_tree* t, const double* x, const double* y,
                            const double* z, const double* q, int32_t degree,
                            int32_t threads, double* qhat)
{
    if (degree < 1 || degree > ORACLE_MAX_DEGREE) return -1;
    const int n1 = degree + 1;
    const int64_t P = (int64_t)n1 * n1 * n1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < t->n_nodes; ++c) {
        double* qh = qhat + c * P;
        for (int64_t k = 0; k < P; ++k) qh[k] = 0.0;
        const double* lo = t->lo + 3 * c;
        const double* hi = t->hi + 3 * c;
        double a1[ORACLE_MAX_DEGREE + 1], a2[ORACLE_MAX_DEGREE + 1], a3[ORACLE_MAX_DEGREE + 1];
        for (int64_t i = t->begin[c]; i < t->begin[c] + t->count[c]; ++i) {
            int64_t j = t->perm[i];
            oracle_lagrange(degree, lo[0], hi[0], x[j], a1);
            oracle_lagrange(degree, lo[1], hi[1], y[j], a2);
            oracle_lagrange(degree, lo[2], hi[2], z[j], a3);
            for (int k1 = 0; k1 < n1; ++k1)
                for (int k2 = 0; k2 < n1; ++k2)
                    for (int k3 = 0; k3 < n1; ++k3)
                        qh[(k1 * n1 + k2) * n1 + k3] += a1[k1] * a2[k2] * a3[k3] * q[j];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Treecode, Algorithm 1 with the MAC of Eq. 13 (readings R3-R5).                         */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    const oracle_tree* bt;   /* target batches */
    const oracle_tree* st;   /* source clusters */
    const double *tx, *ty, *tz;              /* targets, original order */
    const double *sx, *sy, *sz, *sq;         /* sources, original order */
    const double* qhat;                      /* n_nodes(st) * P, or NULL when only listing */
    double theta, kappa;
    int32_t kernel, degree;
    int64_t P;
    double* phi;             /* original target order, or NULL when only listing */
    double* phi_abs;
    /* list recording (may be NULL) */
    int64_t *app, *dir;
    int64_t n_app, n_dir, cap_app, cap_dir;
    int fail;
} cp_ctx;

static void list_push(int64_t** a, int64_t* n, int64_t* cap, int64_t v, int* fail)
{
    if (*n == *cap) {
        int64_t nc = *cap ? 2 * *cap : 256;
        int64_t* p = (int64_t*)realloc(*a, (size_t)nc * sizeof(int64_t));
        if (!p) {
            *fail = 1;
            return;
        }
        *a = p;
        *cap = nc;
    }
    (*a)[(*n)++] = v;
}

/* Batch-cluster approximation, Eq. 11: phi_i += sum_k G(x_i, s_k) qhat_k. */
static void approx_interaction(cp_ctx* c, int64_t B, int64_t C)
{
    const int n1 = c->degree + 1;
    double s1[ORACLE_MAX_DEGREE + 1], s2[ORACLE_MAX_DEGREE + 1], s3[ORACLE_MAX_DEGREE + 1];
    double w[ORACLE_MAX_DEGREE + 1];
    const double* lo = c->st->lo + 3 * C;
    const double* hi = c->st->hi + 3 * C;
    oracle_cheb(c->degree, lo[0], hi[0], s1, w);
    oracle_cheb(c->degree, lo[1], hi[1], s2, w);
    oracle_cheb(c->degree, lo[2], hi[2], s3, w);
    const double* qh = c->qhat + C * c->P;
    for (int64_t i = c->bt->begin[B]; i < c->bt->begin[B] + c->bt->count[B]; ++i) {
        int64_t t = c->bt->perm[i];
        double acc = c->phi[t], acc_abs = c->phi_abs ? c->phi_abs[t] : 0.0;
        for (int k1 = 0; k1 < n1; ++k1)
            for (int k2 = 0; k2 < n1; ++k2)
                for (int k3 = 0; k3 < n1; ++k3) {
                    double g;
                    if (!kernel_G(c->kernel, c->kappa, c->degree, c->tx[t], c->ty[t], c->tz[t],
                                  s1[k1], s2[k2], s3[k3], &g))
                        continue;
                    double term = g * qh[(k1 * n1 + k2) * n1 + k3];
                    acc = acc + term;
                    acc_abs = acc_abs + fabs(term);
                }
        c->phi[t] = acc;
        if (c->phi_abs) c->phi_abs[t] = acc_abs;
    }
}

/* Batch-cluster direct sum, Eq. 9: phi_i += sum_{y_j in C} G(x_i, y_j) q_j. */
static void direct_interaction(cp_ctx* c, int64_t B, int64_t C)
{
    for (int64_t i = c->bt->begin[B]; i < c->bt->begin[B] + c->bt->count[B]; ++i) {
        int64_t t = c->bt->perm[i];
        double acc = c->phi[t], acc_abs = c->phi_abs ? c->phi_abs[t] : 0.0;
        for (int64_t m = c->st->begin[C]; m < c->st->begin[C] + c->st->count[C]; ++m) {
            int64_t j = c->st->perm[m];
            double g;
            if (!kernel_G(c->kernel, c->kappa, c->degree, c->tx[t], c->ty[t], c->tz[t],
                          c->sx[j], c->sy[j], c->sz[j], &g))
                continue;
            double term = g * c->sq[j];
            acc = acc + term;
            acc_abs = acc_abs + fabs(term);
        }
        c->phi[t] = acc;
        if (c->phi_abs) c->phi_abs[t] = acc_abs;
    }
}

/* Where Algorithm 1 puts the pair (batch B, cluster C), from the two conditions of Eq. 13:
 * both hold -> C is approximated for B (Eq. 11); the geometric one holds but C has too few
 * particles to interpolate -> the whole of C is summed directly (reading R5); the geometric
 * one fails -> a leaf C is summed directly (Eq. 9), otherwise its children are examined. */
enum { PAIR_APPROX, PAIR_DIRECT, PAIR_CHILDREN };

static int classify_pair(const cp_ctx* c, int64_t B, int64_t C)
{
    const double* cb = c->bt->center + 3 * B;
    const double* cc = c->st->center + 3 * C;
    double dx = cb[0] - cc[0];
    double dy = cb[1] - cc[1];
    double dz = cb[2] - cc[2];
    double R = sqrt(dx * dx + dy * dy + dz * dz);
    double ratio = (c->bt->radius[B] + c->st->radius[C]) / R;
    int geometric_ok = ratio < c->theta;      /* Eq. 13, first condition (R4) */
    int size_ok = c->P < c->st->count[C];      /* Eq. 13, second condition */
    if (geometric_ok) return size_ok ? PAIR_APPROX : PAIR_DIRECT;
    return c->st->n_children[C] == 0 ? PAIR_DIRECT : PAIR_CHILDREN;
}

/* Algorithm 1 for one batch B: the source tree is examined depth first from the root with
 * an explicit stack (children pushed last to first, so they are examined in stored order);
 * every approximated or directly summed cluster is recorded and summed in that order. */
static void batch_potential(cp_ctx* c, int64_t B)
{
    int32_t depth = 0;
    for (int64_t v = 0; v < c->st->n_nodes; ++v)
        if (c->st->level[v] > depth) depth = c->st->level[v];
    int64_t cap = 8 * ((int64_t)depth + 1) + 1, top = 0;
    int64_t* stack = (int64_t*)malloc((size_t)cap * sizeof(int64_t));
    if (!stack) {
        c->fail = 1;
        return;
    }
    stack[top++] = 0;
    while (top > 0) {
        const int64_t C = stack[--top];
        switch (classify_pair(c, B, C)) {
        case PAIR_APPROX:
            if (c->app) list_push(&c->app, &c->n_app, &c->cap_app, C, &c->fail);
            if (c->phi) approx_interaction(c, B, C);
            break;
        case PAIR_DIRECT:
            if (c->dir) list_push(&c->dir, &c->n_dir, &c->cap_dir, C, &c->fail);
            if (c->phi) direct_interaction(c, B, C);
            break;
        default:
            for (int k = c->st->n_children[C] - 1; k >= 0; --k) stack[top++] = c->st->children[8 * C + k];
            break;
        }
    }
    free(stack);
}

/* Leaves of a tree in DFS order (these are the target batches of a batch tree). */
static int64_t collect_leaves(const oracle_tree* t, int64_t* out)
{
    int64_t m = 0;
    for (int64_t v = 0; v < t->n_nodes; ++v)
        if (t->n_children[v] == 0) {
            if (out) out[m] = v;
            m++;
        }
    return m;
}

int64_t oracle_num_leaves(const oracle_tree* t) { return collect_leaves(t, NULL); }

void oracle_leaves(const oracle_tree* t, int64_t* out) { collect_leaves(t, out); }

/* Interaction lists of every batch (leaf of bt, in DFS order), as CSR arrays.  The caller
 * passes arrays sized by a first call with NULL outputs, which only returns the totals. */
int oracle_lists(const oracle_tree* bt, const oracle_tree* st, double theta, int32_t degree,
                 int64_t* app_off, int64_t* app_ids, int64_t* dir_off, int64_t* dir_ids,
                 int64_t* n_app_total, int64_t* n_dir_total)
{
    int64_t nb = collect_leaves(bt, NULL);
    int64_t* leaves = (int64_t*)malloc((size_t)(nb > 0 ? nb : 1) * sizeof(int64_t));
    if (!leaves) return -2;
    collect_leaves(bt, leaves);
    const int64_t n1 = degree + 1;
    int64_t ta = 0, td = 0;
    if (app_off) app_off[0] = 0;
    if (dir_off) dir_off[0] = 0;
    for (int64_t b = 0; b < nb; ++b) {
        cp_ctx c;
        memset(&c, 0, sizeof(c));
        c.bt = bt;
        c.st = st;
        c.theta = theta;
        c.degree = degree;
        c.P = n1 * n1 * n1;
        c.app = (int64_t*)malloc(256 * sizeof(int64_t));
        c.dir = (int64_t*)malloc(256 * sizeof(int64_t));
        c.cap_app = c.cap_dir = 256;
        if (!c.app || !c.dir) {
            free(c.app);
            free(c.dir);
            free(leaves);
            return -2;
        }
        batch_potential(&c, leaves[b]);
        if (c.fail) {
            free(c.app);
            free(c.dir);
            free(leaves);
            return -2;
        }
        if (app_ids) memcpy(app_ids + ta, c.app, (size_t)c.n_app * sizeof(int64_t));
        if (dir_ids) memcpy(dir_ids + td, c.dir, (size_t)c.n_dir * sizeof(int64_t));
        ta += c.n_app;
        td += c.n_dir;
        if (app_off) app_off[b + 1] = ta;
        if (dir_off) dir_off[b + 1] = td;
        free(c.app);
        free(c.dir);
    }
    free(leaves);
    *n_app_total = ta;
    *n_dir_total = td;
    return 0;
}

static double now_seconds(void)
{
#ifdef _OPENMP
    return omp_get_wtime();
#else
    return 0.0;
#endif
}

/* Algorithm 1's setup for nt targets (tx, ty, tz) and ns sources (sx, sy, sz, sq), which
 * may be different particle sets (Sec. II: the method needs only the target and source
 * positions): the source tree (leaf_size, N_L), the batch tree of the targets (batch_size,
 * N_B) and the modified charges of every source cluster (Eq. 12).  The arrays are read
 * again by oracle_bltc_evaluate and must outlive the handle.  timings (may be NULL)
 * receives setup (trees) and precompute (modified charges) seconds. */
struct oracle_prepared {
    oracle_tree *st, *bt;
    const double *tx, *ty, *tz, *sx, *sy, *sz, *sq;
    int64_t nt, nb;
    int64_t* leaves;
    double* qhat;
    double theta, kappa;
    int32_t kernel, degree;
};

void oracle_bltc_release(oracle_prepared* p)
{
    if (!p) return;
    free(p->leaves);
    free(p->qhat);
    oracle_tree_free(p->st);
    oracle_tree_free(p->bt);
    free(p);
}

int oracle_bltc_prepare(const double* tx, const double* ty, const double* tz, int64_t nt,
                        const double* sx, const double* sy, const double* sz, const double* sq,
                        int64_t ns, double theta, int32_t degree, int32_t leaf_size,
                        int32_t batch_size, int32_t kernel, double kappa, int32_t threads,
                        oracle_prepared** out, double* timings)
{
    *out = NULL;
    if (nt < 1 || ns < 1 || degree < 1 || degree > ORACLE_MAX_DEGREE) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    oracle_prepared* p = (oracle_prepared*)calloc(1, sizeof(oracle_prepared));
    if (!p) return -2;
    double t0 = now_seconds();
    if (oracle_tree_build(sx, sy, sz, ns, leaf_size, &p->st) ||
        oracle_tree_build(tx, ty, tz, nt, batch_size, &p->bt)) {
        oracle_bltc_release(p);
        return -2;
    }
    double t1 = now_seconds();
    const int64_t n1 = degree + 1, P = n1 * n1 * n1;
    p->qhat = (double*)malloc((size_t)(p->st->n_nodes * P) * sizeof(double));
    p->nb = collect_leaves(p->bt, NULL);
    p->leaves = (int64_t*)malloc((size_t)p->nb * sizeof(int64_t));
    if (!p->qhat || !p->leaves) {
        oracle_bltc_release(p);
        return -2;
    }
    collect_leaves(p->bt, p->leaves);
    oracle_modified_charges(p->st, sx, sy, sz, sq, degree, threads, p->qhat);
    double t2 = now_seconds();
    p->tx = tx; p->ty = ty; p->tz = tz;
    p->sx = sx; p->sy = sy; p->sz = sz; p->sq = sq;
    p->nt = nt;
    p->theta = theta;
    p->kappa = kappa;
    p->kernel = kernel;
    p->degree = degree;
    if (timings) {
        timings[0] = t1 - t0;
        timings[1] = t2 - t1;
    }
    *out = p;
    return 0;
}

int64_t oracle_bltc_num_batches(const oracle_prepared* p) { return p ? p->nb : 0; }

/* Algorithm 1's evaluation over the prepared setup: every batch (or only batch_subset, indices
 * into the DFS-ordered leaves of the batch tree; phi of the other targets is left at 0), in
 * parallel over batches.  *seconds (may be NULL) receives the time taken. */
int oracle_bltc_evaluate(const oracle_prepared* p, const int64_t* batch_subset, int64_t n_subset,
                         int32_t threads, double* phi, double* phi_abs, double* seconds)
{
    if (!p) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    double t0 = now_seconds();
    const int64_t n1 = p->degree + 1, P = n1 * n1 * n1;
    for (int64_t i = 0; i < p->nt; ++i) {
        phi[i] = 0.0;
        if (phi_abs) phi_abs[i] = 0.0;
    }
    int64_t todo = batch_subset ? n_subset : p->nb;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t u = 0; u < todo; ++u) {
        int64_t b = batch_subset ? batch_subset[u] : u;
        if (b < 0 || b >= p->nb) {
            bad = 1;
            continue;
        }
        cp_ctx c;
        memset(&c, 0, sizeof(c));
        c.bt = p->bt;
        c.st = p->st;
        c.tx = p->tx;
        c.ty = p->ty;
        c.tz = p->tz;
        c.sx = p->sx;
        c.sy = p->sy;
        c.sz = p->sz;
        c.sq = p->sq;
        c.qhat = p->qhat;
        c.theta = p->theta;
        c.kappa = p->kappa;
        c.kernel = p->kernel;
        c.degree = p->degree;
        c.P = P;
        c.phi = phi;
        c.phi_abs = phi_abs;
        batch_potential(&c, p->leaves[b]);
        if (c.fail) bad = 1;
    }
    if (seconds) *seconds = now_seconds() - t0;
    return bad ? -1 : 0;
}

/* Algorithm 1 for distinct target and source sets: the setup, the evaluation of every batch
 * (or of batch_subset), and the release.  timings receives setup (trees), precompute
 * (modified charges) and compute seconds. */
int oracle_bltc_ts(const double* tx, const double* ty, const double* tz, int64_t nt,
                   const double* sx, const double* sy, const double* sz, const double* sq,
                   int64_t ns, double theta, int32_t degree, int32_t leaf_size,
                   int32_t batch_size, int32_t kernel, double kappa, int32_t threads,
                   const int64_t* batch_subset, int64_t n_subset, double* phi, double* phi_abs,
                   double* timings)
{
    oracle_prepared* p = NULL;
    double tm[2] = {0.0, 0.0}, tc = 0.0;
    int rc = oracle_bltc_prepare(tx, ty, tz, nt, sx, sy, sz, sq, ns, theta, degree, leaf_size,
                                 batch_size, kernel, kappa, threads, &p, tm);
    if (rc) return rc;
    rc = oracle_bltc_evaluate(p, batch_subset, n_subset, threads, phi, phi_abs, &tc);
    if (timings) {
        timings[0] = tm[0];
        timings[1] = tm[1];
        timings[2] = tc;
    }
    oracle_bltc_release(p);
    return rc;
}

/* Algorithm 1 with targets = sources (x, y, z, q), as in all of the paper's runs. */
int oracle_bltc(const double* x, const double* y, const double* z, const double* q, int64_t n,
                double theta, int32_t degree, int32_t leaf_size, int32_t batch_size,
                int32_t kernel, double kappa, int32_t threads, const int64_t* batch_subset,
                int64_t n_subset, double* phi, double* phi_abs, double* timings)
{
    return oracle_bltc_ts(x, y, z, n, x, y, z, q, n, theta, degree, leaf_size, batch_size,
                          kernel, kappa, threads, batch_subset, n_subset, phi, phi_abs, timings);
}

/* ------------------------------------------------------------------------------------ */
/* Cluster-particle variant (the paper's future work, Sec. V): the roles of Algorithm 1    */
/* swapped.  Targets form the clusters, which are interpolated; sources form the batches,  */
/* which are summed exactly.                                                              */
/* ------------------------------------------------------------------------------------ */

/* Per source batch S (a leaf of the source tree, DFS order), Algorithm 1's walk covers the
 * target tree with the same MAC (Eq. 13, here (r_S + r_T)/R < theta and (n+1)^3 < N_T):
 *   - approximated target cluster T: the potential at T's Chebyshev points,
 *       phihat_T[k] += sum_{y_j in S} G(t_k, y_j) q_j,        t_k = (s1[k1], s2[k2], s3[k3]);
 *   - direct (leaf T, or T failing the size test): phi(x_i) += sum_{y_j in S} G(x_i, y_j) q_j
 *     for every target x_i in T.
 * Afterwards every target takes the interpolant of each of its clusters' point potentials,
 *   phi(x_i) += sum_k L_k1(x_i1) L_k2(x_i2) L_k3(x_i3) phihat_T[k]   (Eq. 4-8, exact hits),
 * clusters from the root down.  The direct part of a target is summed over batches S in
 * ascending order, particles in tree order; phihat_T the same way. */
int oracle_bltc_cp(const double* tx, const double* ty, const double* tz, int64_t nt,
                   const double* sx, const double* sy, const double* sz, const double* sq,
                   int64_t ns, double theta, int32_t degree, int32_t leaf_size,
                   int32_t batch_size, int32_t kernel, double kappa, int32_t threads,
                   double* phi, double* phi_abs)
{
    if (nt < 1 || ns < 1 || degree < 1 || degree > ORACLE_MAX_DEGREE) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    oracle_tree *tt = NULL, *st = NULL;
    if (oracle_tree_build(tx, ty, tz, nt, leaf_size, &tt)) return -2;
    if (oracle_tree_build(sx, sy, sz, ns, batch_size, &st)) {
        oracle_tree_free(tt);
        return -2;
    }
    const int n1 = degree + 1;
    const int64_t P = (int64_t)n1 * n1 * n1;
    const int64_t m = tt->n_nodes;
    int rc = -2;
    /* the lists, per source batch: target clusters approximated / summed directly */
    int64_t nb = collect_leaves(st, NULL), na = 0, nd = 0;
    int64_t* sleaves = (int64_t*)malloc((size_t)nb * sizeof(int64_t));
    int64_t* a_off = (int64_t*)malloc((size_t)(nb + 1) * sizeof(int64_t));
    int64_t* d_off = (int64_t*)malloc((size_t)(nb + 1) * sizeof(int64_t));
    int64_t *a_ids = NULL, *d_ids = NULL;
    /* per target node: the batches approximated into it; per target leaf: the batches
     * summed directly (a direct non-leaf cluster passes its batch to all of its leaves) */
    int64_t *ta_off = NULL, *ta_ids = NULL, *td_off = NULL, *td_ids = NULL, *fill = NULL;
    int64_t* leaf_of = NULL;     /* target position -> its leaf */
    double *phat = NULL, *phat_abs = NULL, *near = NULL, *near_abs = NULL;
    if (!sleaves || !a_off || !d_off) goto done;
    collect_leaves(st, sleaves);
    if (oracle_lists(st, tt, theta, degree, NULL, NULL, NULL, NULL, &na, &nd)) goto done;
    a_ids = (int64_t*)malloc((size_t)(na > 0 ? na : 1) * sizeof(int64_t));
    d_ids = (int64_t*)malloc((size_t)(nd > 0 ? nd : 1) * sizeof(int64_t));
    if (!a_ids || !d_ids) goto done;
    if (oracle_lists(st, tt, theta, degree, a_off, a_ids, d_off, d_ids, &na, &nd)) goto done;

    ta_off = (int64_t*)calloc((size_t)(m + 1), sizeof(int64_t));
    td_off = (int64_t*)calloc((size_t)(m + 1), sizeof(int64_t));
    fill = (int64_t*)calloc((size_t)(m + 1), sizeof(int64_t));
    leaf_of = (int64_t*)malloc((size_t)nt * sizeof(int64_t));
    if (!ta_off || !td_off || !fill || !leaf_of) goto done;
    for (int64_t v = 0; v < m; ++v)
        if (tt->n_children[v] == 0)
            for (int64_t i = tt->begin[v]; i < tt->begin[v] + tt->count[v]; ++i) leaf_of[i] = v;
    /* counts */
    int64_t n_td = 0;
    for (int64_t e = 0; e < na; ++e) ta_off[a_ids[e] + 1]++;
    for (int64_t b = 0; b < nb; ++b)
        for (int64_t e = d_off[b]; e < d_off[b + 1]; ++e) {
            const int64_t T = d_ids[e];
            for (int64_t v = T; v < m && (v == T || tt->begin[v] < tt->begin[T] + tt->count[T]); ++v)
                if (tt->n_children[v] == 0) { td_off[v + 1]++; n_td++; }
        }
    for (int64_t v = 0; v < m; ++v) {
        ta_off[v + 1] += ta_off[v];
        td_off[v + 1] += td_off[v];
    }
    ta_ids = (int64_t*)malloc((size_t)(na > 0 ? na : 1) * sizeof(int64_t));
    td_ids = (int64_t*)malloc((size_t)(n_td > 0 ? n_td : 1) * sizeof(int64_t));
    if (!ta_ids || !td_ids) goto done;
    for (int64_t b = 0; b < nb; ++b)          /* ascending b, so every list is ascending */
        for (int64_t e = a_off[b]; e < a_off[b + 1]; ++e) {
            const int64_t T = a_ids[e];
            ta_ids[ta_off[T] + fill[T]++] = b;
        }
    memset(fill, 0, (size_t)(m + 1) * sizeof(int64_t));
    for (int64_t b = 0; b < nb; ++b)
        for (int64_t e = d_off[b]; e < d_off[b + 1]; ++e) {
            const int64_t T = d_ids[e];
            for (int64_t v = T; v < m && (v == T || tt->begin[v] < tt->begin[T] + tt->count[T]); ++v)
                if (tt->n_children[v] == 0) td_ids[td_off[v] + fill[v]++] = b;
        }

    /* potentials at the Chebyshev points of every approximated target cluster */
    phat = (double*)calloc((size_t)(m * P), sizeof(double));
    phat_abs = (double*)calloc((size_t)(m * P), sizeof(double));
    if (!phat || !phat_abs) goto done;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t T = 0; T < m; ++T) {
        if (ta_off[T + 1] == ta_off[T]) continue;
        double s1[ORACLE_MAX_DEGREE + 1], s2[ORACLE_MAX_DEGREE + 1], s3[ORACLE_MAX_DEGREE + 1];
        double w[ORACLE_MAX_DEGREE + 1];
        oracle_cheb(degree, tt->lo[3 * T], tt->hi[3 * T], s1, w);
        oracle_cheb(degree, tt->lo[3 * T + 1], tt->hi[3 * T + 1], s2, w);
        oracle_cheb(degree, tt->lo[3 * T + 2], tt->hi[3 * T + 2], s3, w);
        for (int k1 = 0; k1 < n1; ++k1)
            for (int k2 = 0; k2 < n1; ++k2)
                for (int k3 = 0; k3 < n1; ++k3) {
                    double acc = 0.0, acc_abs = 0.0;
                    for (int64_t e = ta_off[T]; e < ta_off[T + 1]; ++e) {
                        const int64_t S = sleaves[ta_ids[e]];
                        for (int64_t mm = st->begin[S]; mm < st->begin[S] + st->count[S]; ++mm) {
                            const int64_t j = st->perm[mm];
                            double g;
                            if (!kernel_G(kernel, kappa, degree, s1[k1], s2[k2], s3[k3], sx[j], sy[j],
                                          sz[j], &g))
                                continue;
                            acc = acc + g * sq[j];
                            acc_abs = acc_abs + fabs(g * sq[j]);
                        }
                    }
                    phat[T * P + (k1 * n1 + k2) * n1 + k3] = acc;
                    phat_abs[T * P + (k1 * n1 + k2) * n1 + k3] = acc_abs;
                }
    }
    /* direct part, then the interpolants of the target's clusters from the root down */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nt; ++i) {
        const int64_t L = leaf_of[i];
        const int64_t t = tt->perm[i];
        double acc = 0.0, acc_abs = 0.0;
        for (int64_t e = td_off[L]; e < td_off[L + 1]; ++e) {
            const int64_t S = sleaves[td_ids[e]];
            for (int64_t mm = st->begin[S]; mm < st->begin[S] + st->count[S]; ++mm) {
                const int64_t j = st->perm[mm];
                double g;
                if (!kernel_G(kernel, kappa, degree, tx[t], ty[t], tz[t], sx[j], sy[j], sz[j], &g))
                    continue;
                acc = acc + g * sq[j];
                acc_abs = acc_abs + fabs(g * sq[j]);
            }
        }
        int64_t chain[128];
        int depth = 0;
        for (int64_t v = L; v >= 0 && depth < 128; v = tt->parent[v]) chain[depth++] = v;
        for (int d = depth - 1; d >= 0; --d) {
            const int64_t T = chain[d];
            if (ta_off[T + 1] == ta_off[T]) continue;
            double a1[ORACLE_MAX_DEGREE + 1], a2[ORACLE_MAX_DEGREE + 1], a3[ORACLE_MAX_DEGREE + 1];
            oracle_lagrange(degree, tt->lo[3 * T], tt->hi[3 * T], tx[t], a1);
            oracle_lagrange(degree, tt->lo[3 * T + 1], tt->hi[3 * T + 1], ty[t], a2);
            oracle_lagrange(degree, tt->lo[3 * T + 2], tt->hi[3 * T + 2], tz[t], a3);
            for (int k1 = 0; k1 < n1; ++k1)
                for (int k2 = 0; k2 < n1; ++k2)
                    for (int k3 = 0; k3 < n1; ++k3) {
                        const int64_t k = (k1 * n1 + k2) * n1 + k3;
                        const double l = a1[k1] * a2[k2] * a3[k3];
                        acc = acc + l * phat[T * P + k];
                        acc_abs = acc_abs + fabs(l) * phat_abs[T * P + k];
                    }
        }
        phi[t] = acc;
        if (phi_abs) phi_abs[t] = acc_abs;
    }
    rc = 0;
done:
    free(sleaves); free(a_off); free(d_off); free(a_ids); free(d_ids);
    free(ta_off); free(ta_ids); free(td_off); free(td_ids); free(fill); free(leaf_of);
    free(phat); free(phat_abs); free(near); free(near_abs);
    oracle_tree_free(tt);
    oracle_tree_free(st);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Cluster-cluster variant (dual tree traversal, the paper's future work, Sec. V).         */
/* ------------------------------------------------------------------------------------ */

/* Reading (the paper names the variant but does not define it).  Both sides are trees:
 * sources with leaf_size (N_L), targets with batch_size (N_B).  DualTraversal(T, S) starts
 * at the two roots:
 *   if (r_T + r_S)/R < theta (Eq. 13's geometric test):
 *       P < N_T and P < N_S  -> CC: phihat_T[k] += sum_k' G(t_k, s_k') qhat_S[k']
 *       P < N_T only         -> CP: phihat_T[k] += sum_{y_j in S} G(t_k, y_j) q_j
 *       P < N_S only         -> PC: phi(x_i) += sum_k' G(x_i, s_k') qhat_S[k'],  x_i in T
 *       neither              -> PP: phi(x_i) += sum_{y_j in S} G(x_i, y_j) q_j, x_i in T
 *   else if T and S are leaves -> PP
 *   else split one side, children in stored order: T if S is a leaf, or if T is not a leaf and
 *       r_T >= r_S; S otherwise.
 * Finally phi(x_i) += sum_k L_k1 L_k2 L_k3 (x_i) phihat_T[k] for every target cluster T holding
 * x_i (Eq. 4-8, exact hits), root first.  Per target the PC and PP terms are summed for its
 * clusters root first, each cluster's interactions in traversal order. */
typedef struct {
    int64_t *t, *s;
    int64_t n, cap;
} pair_list;

static int pair_push(pair_list* l, int64_t t, int64_t s)
{
    if (l->n == l->cap) {
        int64_t nc = l->cap ? 2 * l->cap : 1024;
        int64_t* a = (int64_t*)realloc(l->t, (size_t)nc * sizeof(int64_t));
        if (!a) return -1;
        l->t = a;
        a = (int64_t*)realloc(l->s, (size_t)nc * sizeof(int64_t));
        if (!a) return -1;
        l->s = a;
        l->cap = nc;
    }
    l->t[l->n] = t;
    l->s[l->n] = s;
    l->n++;
    return 0;
}

typedef struct {
    const oracle_tree *tt, *st;
    double theta;
    int64_t P;
    pair_list cc, cp, pc, pp;
    int fail;
} dual_ctx;

static void dual_traverse(dual_ctx* c, int64_t T, int64_t S)
{
    const double* ct = c->tt->center + 3 * T;
    const double* cs = c->st->center + 3 * S;
    double dx = ct[0] - cs[0];
    double dy = ct[1] - cs[1];
    double dz = ct[2] - cs[2];
    double R = sqrt(dx * dx + dy * dy + dz * dz);
    double ratio = (c->tt->radius[T] + c->st->radius[S]) / R;
    const int t_leaf = c->tt->n_children[T] == 0, s_leaf = c->st->n_children[S] == 0;
    if (ratio < c->theta) {
        const int tc = c->P < c->tt->count[T], sc = c->P < c->st->count[S];
        pair_list* l = tc ? (sc ? &c->cc : &c->cp) : (sc ? &c->pc : &c->pp);
        if (pair_push(l, T, S)) c->fail = 1;
    } else if (t_leaf && s_leaf) {
        if (pair_push(&c->pp, T, S)) c->fail = 1;
    } else if (s_leaf || (!t_leaf && c->tt->radius[T] >= c->st->radius[S])) {
        for (int k = 0; k < c->tt->n_children[T]; ++k) dual_traverse(c, c->tt->children[8 * T + k], S);
    } else {
        for (int k = 0; k < c->st->n_children[S]; ++k) dual_traverse(c, T, c->st->children[8 * S + k]);
    }
}

/* The four interaction lists of the dual traversal, in traversal order (pairs of target and
 * source node ids).  Arrays are malloc'ed; the caller frees them with free(). */
int oracle_dual_lists(const oracle_tree* tt, const oracle_tree* st, double theta, int32_t degree,
                      int64_t* n_out, int64_t** t_out, int64_t** s_out)
{
    dual_ctx c;
    memset(&c, 0, sizeof(c));
    c.tt = tt;
    c.st = st;
    c.theta = theta;
    c.P = (int64_t)(degree + 1) * (degree + 1) * (degree + 1);
    dual_traverse(&c, 0, 0);
    pair_list* ls[4] = {&c.cc, &c.cp, &c.pc, &c.pp};
    for (int i = 0; i < 4; ++i) {
        n_out[i] = ls[i]->n;
        t_out[i] = ls[i]->t;
        s_out[i] = ls[i]->s;
    }
    return c.fail ? -2 : 0;
}

/* Copies the four lists (CC, CP, PC, PP) into caller arrays sized by a first call with NULL
 * arrays, which only returns the counts. */
int oracle_dual_lists_export(const oracle_tree* tt, const oracle_tree* st, double theta,
                             int32_t degree, int64_t* counts, int64_t* t_ids, int64_t* s_ids)
{
    int64_t n[4];
    int64_t *t[4], *s[4];
    int rc = oracle_dual_lists(tt, st, theta, degree, n, t, s);
    int64_t o = 0;
    for (int i = 0; i < 4; ++i) {
        counts[i] = n[i];
        if (t_ids && s_ids) {
            memcpy(t_ids + o, t[i], (size_t)n[i] * sizeof(int64_t));
            memcpy(s_ids + o, s[i], (size_t)n[i] * sizeof(int64_t));
        }
        o += n[i];
        free(t[i]);
        free(s[i]);
    }
    return rc;
}

int oracle_bltc_cc(const double* tx, const double* ty, const double* tz, int64_t nt,
                   const double* sx, const double* sy, const double* sz, const double* sq,
                   int64_t ns, double theta, int32_t degree, int32_t leaf_size,
                   int32_t batch_size, int32_t kernel, double kappa, int32_t threads,
                   double* phi, double* phi_abs)
{
    if (nt < 1 || ns < 1 || degree < 1 || degree > ORACLE_MAX_DEGREE) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    oracle_tree *tt = NULL, *st = NULL;
    if (oracle_tree_build(sx, sy, sz, ns, leaf_size, &st)) return -2;
    if (oracle_tree_build(tx, ty, tz, nt, batch_size, &tt)) {
        oracle_tree_free(st);
        return -2;
    }
    const int n1 = degree + 1;
    const int64_t P = (int64_t)n1 * n1 * n1;
    const int64_t mt = tt->n_nodes, ms = st->n_nodes;
    int rc = -2;
    int64_t n[4] = {0, 0, 0, 0};
    int64_t *lt[4] = {NULL, NULL, NULL, NULL}, *ls[4] = {NULL, NULL, NULL, NULL};
    /* per target node, its interactions of each kind (CSR over target nodes, traversal order) */
    int64_t *off[4] = {NULL, NULL, NULL, NULL}, *ids[4] = {NULL, NULL, NULL, NULL};
    double *qhat = NULL, *phat = NULL, *phat_abs = NULL;
    int64_t* leaf_of = NULL;
    if (oracle_dual_lists(tt, st, theta, degree, n, lt, ls)) goto done;
    for (int i = 0; i < 4; ++i) {
        off[i] = (int64_t*)calloc((size_t)(mt + 1), sizeof(int64_t));
        ids[i] = (int64_t*)malloc((size_t)(n[i] > 0 ? n[i] : 1) * sizeof(int64_t));
        if (!off[i] || !ids[i]) goto done;
        for (int64_t e = 0; e < n[i]; ++e) off[i][lt[i][e] + 1]++;
        for (int64_t v = 0; v < mt; ++v) off[i][v + 1] += off[i][v];
        int64_t* fill = (int64_t*)calloc((size_t)(mt + 1), sizeof(int64_t));
        if (!fill) goto done;
        for (int64_t e = 0; e < n[i]; ++e) ids[i][off[i][lt[i][e]] + fill[lt[i][e]]++] = ls[i][e];
        free(fill);
    }
    qhat = (double*)malloc((size_t)(ms * P) * sizeof(double));
    phat = (double*)calloc((size_t)(mt * P), sizeof(double));
    phat_abs = (double*)calloc((size_t)(mt * P), sizeof(double));
    leaf_of = (int64_t*)malloc((size_t)nt * sizeof(int64_t));
    if (!qhat || !phat || !phat_abs || !leaf_of) goto done;
    oracle_modified_charges(st, sx, sy, sz, sq, degree, threads, qhat);
    for (int64_t v = 0; v < mt; ++v)
        if (tt->n_children[v] == 0)
            for (int64_t i = tt->begin[v]; i < tt->begin[v] + tt->count[v]; ++i) leaf_of[i] = v;

    /* point potentials of the target clusters: CC terms, then CP terms */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t T = 0; T < mt; ++T) {
        if (off[0][T + 1] == off[0][T] && off[1][T + 1] == off[1][T]) continue;
        double t1[ORACLE_MAX_DEGREE + 1], t2[ORACLE_MAX_DEGREE + 1], t3[ORACLE_MAX_DEGREE + 1];
        double w[ORACLE_MAX_DEGREE + 1];
        oracle_cheb(degree, tt->lo[3 * T], tt->hi[3 * T], t1, w);
        oracle_cheb(degree, tt->lo[3 * T + 1], tt->hi[3 * T + 1], t2, w);
        oracle_cheb(degree, tt->lo[3 * T + 2], tt->hi[3 * T + 2], t3, w);
        for (int k1 = 0; k1 < n1; ++k1)
            for (int k2 = 0; k2 < n1; ++k2)
                for (int k3 = 0; k3 < n1; ++k3) {
                    double acc = 0.0, acc_abs = 0.0;
                    for (int64_t e = off[0][T]; e < off[0][T + 1]; ++e) {
                        const int64_t S = ids[0][e];
                        double s1[ORACLE_MAX_DEGREE + 1], s2[ORACLE_MAX_DEGREE + 1], s3[ORACLE_MAX_DEGREE + 1];
                        oracle_cheb(degree, st->lo[3 * S], st->hi[3 * S], s1, w);
                        oracle_cheb(degree, st->lo[3 * S + 1], st->hi[3 * S + 1], s2, w);
                        oracle_cheb(degree, st->lo[3 * S + 2], st->hi[3 * S + 2], s3, w);
                        for (int m1 = 0; m1 < n1; ++m1)
                            for (int m2 = 0; m2 < n1; ++m2)
                                for (int m3 = 0; m3 < n1; ++m3) {
                                    double g;
                                    if (!kernel_G(kernel, kappa, degree, t1[k1], t2[k2], t3[k3], s1[m1],
                                                  s2[m2], s3[m3], &g))
                                        continue;
                                    const double term = g * qhat[S * P + (m1 * n1 + m2) * n1 + m3];
                                    acc = acc + term;
                                    acc_abs = acc_abs + fabs(term);
                                }
                    }
                    for (int64_t e = off[1][T]; e < off[1][T + 1]; ++e) {
                        const int64_t S = ids[1][e];
                        for (int64_t mm = st->begin[S]; mm < st->begin[S] + st->count[S]; ++mm) {
                            const int64_t j = st->perm[mm];
                            double g;
                            if (!kernel_G(kernel, kappa, degree, t1[k1], t2[k2], t3[k3], sx[j], sy[j],
                                          sz[j], &g))
                                continue;
                            acc = acc + g * sq[j];
                            acc_abs = acc_abs + fabs(g * sq[j]);
                        }
                    }
                    phat[T * P + (k1 * n1 + k2) * n1 + k3] = acc;
                    phat_abs[T * P + (k1 * n1 + k2) * n1 + k3] = acc_abs;
                }
    }
    /* per target: PC and PP terms of its clusters root first, then the interpolants */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nt; ++i) {
        const int64_t t = tt->perm[i];
        int64_t chain[128];
        int depth = 0;
        for (int64_t v = leaf_of[i]; v >= 0 && depth < 128; v = tt->parent[v]) chain[depth++] = v;
        double acc = 0.0, acc_abs = 0.0;
        for (int d = depth - 1; d >= 0; --d) {
            const int64_t T = chain[d];
            for (int64_t e = off[2][T]; e < off[2][T + 1]; ++e) {        /* PC */
                const int64_t S = ids[2][e];
                double s1[ORACLE_MAX_DEGREE + 1], s2[ORACLE_MAX_DEGREE + 1], s3[ORACLE_MAX_DEGREE + 1];
                double w[ORACLE_MAX_DEGREE + 1];
                oracle_cheb(degree, st->lo[3 * S], st->hi[3 * S], s1, w);
                oracle_cheb(degree, st->lo[3 * S + 1], st->hi[3 * S + 1], s2, w);
                oracle_cheb(degree, st->lo[3 * S + 2], st->hi[3 * S + 2], s3, w);
                for (int m1 = 0; m1 < n1; ++m1)
                    for (int m2 = 0; m2 < n1; ++m2)
                        for (int m3 = 0; m3 < n1; ++m3) {
                            double g;
                            if (!kernel_G(kernel, kappa, degree, tx[t], ty[t], tz[t], s1[m1], s2[m2],
                                          s3[m3], &g))
                                continue;
                            const double term = g * qhat[S * P + (m1 * n1 + m2) * n1 + m3];
                            acc = acc + term;
                            acc_abs = acc_abs + fabs(term);
                        }
            }
            for (int64_t e = off[3][T]; e < off[3][T + 1]; ++e) {        /* PP */
                const int64_t S = ids[3][e];
                for (int64_t mm = st->begin[S]; mm < st->begin[S] + st->count[S]; ++mm) {
                    const int64_t j = st->perm[mm];
                    double g;
                    if (!kernel_G(kernel, kappa, degree, tx[t], ty[t], tz[t], sx[j], sy[j], sz[j], &g))
                        continue;
                    acc = acc + g * sq[j];
                    acc_abs = acc_abs + fabs(g * sq[j]);
                }
            }
        }
        for (int d = depth - 1; d >= 0; --d) {
            const int64_t T = chain[d];
            if (off[0][T + 1] == off[0][T] && off[1][T + 1] == off[1][T]) continue;
            double a1[ORACLE_MAX_DEGREE + 1], a2[ORACLE_MAX_DEGREE + 1], a3[ORACLE_MAX_DEGREE + 1];
            oracle_lagrange(degree, tt->lo[3 * T], tt->hi[3 * T], tx[t], a1);
            oracle_lagrange(degree, tt->lo[3 * T + 1], tt->hi[3 * T + 1], ty[t], a2);
            oracle_lagrange(degree, tt->lo[3 * T + 2], tt->hi[3 * T + 2], tz[t], a3);
            for (int k1 = 0; k1 < n1; ++k1)
                for (int k2 = 0; k2 < n1; ++k2)
                    for (int k3 = 0; k3 < n1; ++k3) {
                        const int64_t k = (k1 * n1 + k2) * n1 + k3;
                        const double l = a1[k1] * a2[k2] * a3[k3];
                        acc = acc + l * phat[T * P + k];
                        acc_abs = acc_abs + fabs(l) * phat_abs[T * P + k];
                    }
        }
        phi[t] = acc;
        if (phi_abs) phi_abs[t] = acc_abs;
    }
    rc = 0;
done:
    for (int i = 0; i < 4; ++i) {
        free(lt[i]); free(ls[i]); free(off[i]); free(ids[i]);
    }
    free(qhat); free(phat); free(phat_abs); free(leaf_of);
    oracle_tree_free(tt);
    oracle_tree_free(st);
    return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Barycentric Hermite treecode (the paper's future work, Sec. V).                         */
/* ------------------------------------------------------------------------------------ */

/* Reading (the paper names the method without defining it).  On the n+1 Chebyshev points of
 * Eq. 6 the Hermite interpolant of a function f of one variable is
 *     p(y) = sum_k f(s_k) H_k(y) + f'(s_k) K_k(y),
 *     H_k(y) = (1 - 2 L_k'(s_k) (y - s_k)) L_k(y)^2,   K_k(y) = (y - s_k) L_k(y)^2,
 * with L_k of Eq. 4 and L_k'(s_k) = sum_{j != k} 1/(s_k - s_j); it reproduces polynomials of
 * degree 2n+1.  The tensor product in three variables needs the 8 mixed derivatives
 * D^a = d^{a1}/dy1 d^{a2}/dy2 d^{a3}/dy3, a in {0,1}^3 (index a1*4 + a2*2 + a3), so that
 *     phi(x_i) ~ sum_k sum_a D^a G(x_i, s_k) qhat^a_k,
 *     qhat^a_k = sum_{y_j in C} q_j B^{a1}_{k1}(y_j1) B^{a2}_{k2}(y_j2) B^{a3}_{k3}(y_j3),
 * B^0 = H, B^1 = K.  An exact hit y = s_m (Sec. II-C) gives H = e_m, K = 0.  The MAC is
 * Eq. 13 with the size test 8(n+1)^3 < N_C (the approximation evaluates 8 terms per point).
 * For a radial kernel G(r), r = |x - y|, d = x - y: D^a G = prod_{l: a_l = 1} d_l * G_|a|(r)
 * with G_0 = G and G_{m+1}(r) = -G_m'(r)/r. */
static void hermite_factors(int32_t degree, double lo, double hi, double y, double* h, double* k)
{
    double s[ORACLE_MAX_DEGREE + 1], w[ORACLE_MAX_DEGREE + 1], l[ORACLE_MAX_DEGREE + 1];
    oracle_cheb(degree, lo, hi, s, w);
    for (int m = 0; m <= degree; ++m) {
        if (fabs(y - s[m]) < DBL_MIN) {
            for (int j = 0; j <= degree; ++j) {
                h[j] = (j == m) ? 1.0 : 0.0;
                k[j] = 0.0;
            }
            return;
        }
    }
    oracle_lagrange(degree, lo, hi, y, l);
    for (int j = 0; j <= degree; ++j) {
        double dl = 0.0;
        for (int m = 0; m <= degree; ++m)
            if (m != j) dl = dl + 1.0 / (s[j] - s[m]);
        const double l2 = l[j] * l[j];
        h[j] = (1.0 - 2.0 * dl * (y - s[j])) * l2;
        k[j] = (y - s[j]) * l2;
    }
}

void oracle_hermite_factors(int32_t degree, double lo, double hi, double y, double* h, double* k)
{
    hermite_factors(degree, lo, hi, y, h, k);
}

/* D^a G(x, y) for the 8 a in {0,1}^3; returns 0 when r^2 == 0 (pair skipped, reading R1).
 * The polynomial test kernel is prod_l (1 + x_l y_l / 2)^kdeg. */
static int kernel_dG(int kernel, double kappa, int kdeg, double tx, double ty, double tz,
                     double sx, double sy, double sz, double* out)
{
    const double d[3] = {tx - sx, ty - sy, tz - sz};
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0) {
        return 0;
    }
    if (kernel == ORACLE_KERNEL_POLY) {
        const double xs[3] = {tx, ty, tz}, ys[3] = {sx, sy, sz};
        double f[3], df[3];
        for (int l = 0; l < 3; ++l) {
            const double b = 1.0 + 0.5 * xs[l] * ys[l];
            double pm1 = 1.0;
            for (int m = 0; m < kdeg - 1; ++m) pm1 = pm1 * b;
            f[l] = pm1 * b;
            df[l] = (double)kdeg * pm1 * 0.5 * xs[l];
        }
        for (int a = 0; a < 8; ++a)
            out[a] = ((a & 4) ? df[0] : f[0]) * ((a & 2) ? df[1] : f[1]) * ((a & 1) ? df[2] : f[2]);
        return 1;
    }
    double g[4];
    if (kernel == ORACLE_KERNEL_SOFT) {
        const double u = r2 + kappa * kappa;         /* (r^2 + eps^2) */
        const double v = 1.0 / sqrt(u);
        g[0] = v;
        g[1] = v / u;
        g[2] = 3.0 * v / (u * u);
        g[3] = 15.0 * v / (u * u * u);
    } else {
        const double r = sqrt(r2);
        const double e = (kernel == ORACLE_KERNEL_YUKAWA) ? exp(-kappa * r) : 1.0;
        const double kr = (kernel == ORACLE_KERNEL_YUKAWA) ? kappa * r : 0.0;
        g[0] = e / r;
        g[1] = e * (1.0 + kr) / (r * r2);
        g[2] = e * (3.0 + 3.0 * kr + kr * kr) / (r * r2 * r2);
        g[3] = e * (15.0 + 15.0 * kr + 6.0 * kr * kr + kr * kr * kr) / (r * r2 * r2 * r2);
    }
    for (int a = 0; a < 8; ++a) {
        const int m = ((a >> 2) & 1) + ((a >> 1) & 1) + (a & 1);
        double p = g[m];
        if (a & 4) p = p * d[0];
        if (a & 2) p = p * d[1];
        if (a & 1) p = p * d[2];
        out[a] = p;
    }
    return 1;
}

int oracle_kernel_dG(int32_t kernel, double kappa, int32_t kdeg, const double* x, const double* y,
                     double* out)
{
    return kernel_dG(kernel, kappa, kdeg, x[0], x[1], x[2], y[0], y[1], y[2], out);
}

/* Hermite modified charges of every cluster: [n_nodes][8][(n+1)^3], a-major, k in C order. */
int oracle_hermite_charges(const oracle_tree* t, const double* x, const double* y, const double* z,
                           const double* q, int32_t degree, int32_t threads, double* qh)
{
    if (degree < 1 || degree > ORACLE_MAX_DEGREE) return -1;
    const int n1 = degree + 1;
    const int64_t P = (int64_t)n1 * n1 * n1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#else
    (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < t->n_nodes; ++c) {
        double* out = qh + c * 8 * P;
        for (int64_t k = 0; k < 8 * P; ++k) out[k] = 0.0;
        double h[3][ORACLE_MAX_DEGREE + 1], kk[3][ORACLE_MAX_DEGREE + 1];
        for (int64_t i = t->begin[c]; i < t->begin[c] + t->count[c]; ++i) {
            const int64_t j = t->perm[i];
            const double yv[3] = {x[j], y[j], z[j]};
            for (int d = 0; d < 3; ++d)
                hermite_factors(degree, t->lo[3 * c + d], t->hi[3 * c + d], yv[d], h[d], kk[d]);
            for (int a = 0; a < 8; ++a) {
                const double* f1 = (a & 4) ? kk[0] : h[0];
                const double* f2 = (a & 2) ? kk[1] : h[1];
                const double* f3 = (a & 1) ? kk[2] : h[2];
                for (int k1 = 0; k1 < n1; ++k1)
                    for (int k2 = 0; k2 < n1; ++k2)
                        for (int k3 = 0; k3 < n1; ++k3)
                            out[a * P + (k1 * n1 + k2) * n1 + k3] += f1[k1] * f2[k2] * f3[k3] * q[j];
            }
        }
    }
    return 0;
}

typedef struct {
    const oracle_tree *bt, *st;
    const double *x, *y, *z, *q;
    const double* qh;
    double theta, kappa;
    int32_t kernel, degree;
    int64_t P;
    double *phi, *phi_abs;
} herm_ctx;

static void herm_potential(herm_ctx* c, int64_t B, int64_t C)
{
    const double* cb = c->bt->center + 3 * B;
    const double* cc = c->st->center + 3 * C;
    double dx = cb[0] - cc[0];
    double dy = cb[1] - cc[1];
    double dz = cb[2] - cc[2];
    double R = sqrt(dx * dx + dy * dy + dz * dz);
    double ratio = (c->bt->radius[B] + c->st->radius[C]) / R;
    const int geometric_ok = ratio < c->theta;
    const int size_ok = 8 * c->P < c->st->count[C];
    const int n1 = c->degree + 1;
    if (geometric_ok && size_ok) {
        double s1[ORACLE_MAX_DEGREE + 1], s2[ORACLE_MAX_DEGREE + 1], s3[ORACLE_MAX_DEGREE + 1];
        double w[ORACLE_MAX_DEGREE + 1];
        oracle_cheb(c->degree, c->st->lo[3 * C], c->st->hi[3 * C], s1, w);
        oracle_cheb(c->degree, c->st->lo[3 * C + 1], c->st->hi[3 * C + 1], s2, w);
        oracle_cheb(c->degree, c->st->lo[3 * C + 2], c->st->hi[3 * C + 2], s3, w);
        const double* qh = c->qh + C * 8 * c->P;
        for (int64_t i = c->bt->begin[B]; i < c->bt->begin[B] + c->bt->count[B]; ++i) {
            const int64_t t = c->bt->perm[i];
            double acc = c->phi[t], acc_abs = c->phi_abs ? c->phi_abs[t] : 0.0;
            for (int k1 = 0; k1 < n1; ++k1)
                for (int k2 = 0; k2 < n1; ++k2)
                    for (int k3 = 0; k3 < n1; ++k3) {
                        double dg[8];
                        if (!kernel_dG(c->kernel, c->kappa, 2 * c->degree + 1, c->x[t], c->y[t], c->z[t],
                                       s1[k1], s2[k2], s3[k3], dg))
                            continue;
                        const int64_t k = (k1 * n1 + k2) * n1 + k3;
                        for (int a = 0; a < 8; ++a) {
                            const double term = dg[a] * qh[a * c->P + k];
                            acc = acc + term;
                            acc_abs = acc_abs + fabs(term);
                        }
                    }
            c->phi[t] = acc;
            if (c->phi_abs) c->phi_abs[t] = acc_abs;
        }
    } else if (!geometric_ok && c->st->n_children[C] != 0) {
        for (int k = 0; k < c->st->n_children[C]; ++k) herm_potential(c, B, c->st->children[8 * C + k]);
    } else {
        for (int64_t i = c->bt->begin[B]; i < c->bt->begin[B] + c->bt->count[B]; ++i) {
            const int64_t t = c->bt->perm[i];
            double acc = c->phi[t], acc_abs = c->phi_abs ? c->phi_abs[t] : 0.0;
            for (int64_t m = c->st->begin[C]; m < c->st->begin[C] + c->st->count[C]; ++m) {
                const int64_t j = c->st->perm[m];
                double dg[8];
                if (!kernel_dG(c->kernel, c->kappa, 2 * c->degree + 1, c->x[t], c->y[t], c->z[t],
                               c->x[j], c->y[j], c->z[j], dg))
                    continue;
                const double term = dg[0] * c->q[j];
                acc = acc + term;
                acc_abs = acc_abs + fabs(term);
            }
            c->phi[t] = acc;
            if (c->phi_abs) c->phi_abs[t] = acc_abs;
        }
    }
}

/* The Hermite treecode, targets = sources: Algorithm 1 with the Hermite far field above. */
int oracle_bltc_hermite(const double* x, const double* y, const double* z, const double* q, int64_t n,
                        double theta, int32_t degree, int32_t leaf_size, int32_t batch_size,
                        int32_t kernel, double kappa, int32_t threads, double* phi, double* phi_abs)
{
    if (n < 1 || degree < 1 || degree > ORACLE_MAX_DEGREE) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    oracle_tree *st = NULL, *bt = NULL;
    if (oracle_tree_build(x, y, z, n, leaf_size, &st)) return -2;
    if (oracle_tree_build(x, y, z, n, batch_size, &bt)) {
        oracle_tree_free(st);
        return -2;
    }
    const int64_t n1 = degree + 1, P = n1 * n1 * n1;
    double* qh = (double*)malloc((size_t)(st->n_nodes * 8 * P) * sizeof(double));
    int64_t nb = collect_leaves(bt, NULL);
    int64_t* leaves = (int64_t*)malloc((size_t)nb * sizeof(int64_t));
    if (!qh || !leaves) {
        free(qh);
        free(leaves);
        oracle_tree_free(st);
        oracle_tree_free(bt);
        return -2;
    }
    oracle_hermite_charges(st, x, y, z, q, degree, threads, qh);
    collect_leaves(bt, leaves);
    for (int64_t i = 0; i < n; ++i) {
        phi[i] = 0.0;
        if (phi_abs) phi_abs[i] = 0.0;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nb; ++b) {
        herm_ctx c;
        memset(&c, 0, sizeof(c));
        c.bt = bt;
        c.st = st;
        c.x = x;
        c.y = y;
        c.z = z;
        c.q = q;
        c.qh = qh;
        c.theta = theta;
        c.kappa = kappa;
        c.kernel = kernel;
        c.degree = degree;
        c.P = P;
        c.phi = phi;
        c.phi_abs = phi_abs;
        herm_potential(&c, leaves[b], 0);
    }
    free(qh);
    free(leaves);
    oracle_tree_free(st);
    oracle_tree_free(bt);
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
