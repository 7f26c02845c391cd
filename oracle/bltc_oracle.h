/*
 * bltc_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure only).
 *
 * This header belongs to oracle/ alone.  The CUDA library neither includes it nor shares
 * any of its definitions; tests reach both through their own Python bindings.
 */
#ifndef BLTC_ORACLE_H
#define BLTC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_MAX_DEGREE 32

enum { ORACLE_KERNEL_COULOMB = 0, ORACLE_KERNEL_YUKAWA = 1, ORACLE_KERNEL_POLY = 2,
       ORACLE_KERNEL_SOFT = 3 };

typedef struct oracle_tree oracle_tree;

/* Eq. 1 with the kernels of Eq. 2; pairs with r^2 == 0 are skipped. */
int oracle_direct_sum(const double* tx, const double* ty, const double* tz, int64_t nt,
                      const double* sx, const double* sy, const double* sz, const double* sq,
                      int64_t ns, int32_t kernel, double kappa, int32_t degree,
                      int32_t threads, double* phi, double* phi_abs);

/* Sec. II-D tree of clusters (or batches) with the Sec. III-A aspect-ratio rule. */
int oracle_tree_build(const double* x, const double* y, const double* z, int64_t n,
                      int32_t max_leaf, oracle_tree** out);
void oracle_tree_free(oracle_tree* t);
int64_t oracle_tree_num_nodes(const oracle_tree* t);
void oracle_tree_export(const oracle_tree* t, int64_t* perm, int64_t* begin, int64_t* count,
                        int32_t* parent, int32_t* level, int32_t* n_children,
                        int32_t* children, double* lo, double* hi, double* center,
                        double* radius);
int64_t oracle_num_leaves(const oracle_tree* t);
void oracle_leaves(const oracle_tree* t, int64_t* out);

/* Eq. 6-7 and Eq. 4-5 with the Sec. II-C exact-hit rule. */
void oracle_cheb(int32_t degree, double lo, double hi, double* s, double* w);
void oracle_lagrange(int32_t degree, double lo, double hi, double y, double* a);

/* Eq. 12 for every node of the tree. */
int oracle_modified_charges(const oracle_tree* t, const double* x, const double* y,
                            const double* z, const double* q, int32_t degree,
                            int32_t threads, double* qhat);

/* Algorithm 1's walk of every batch, recording the lists only. */
int oracle_lists(const oracle_tree* bt, const oracle_tree* st, double theta, int32_t degree,
                 int64_t* app_off, int64_t* app_ids, int64_t* dir_off, int64_t* dir_ids,
                 int64_t* n_app_total, int64_t* n_dir_total);

/* Algorithm 1 end to end (targets = sources). */
int oracle_bltc(const double* x, const double* y, const double* z, const double* q, int64_t n,
                double theta, int32_t degree, int32_t leaf_size, int32_t batch_size,
                int32_t kernel, double kappa, int32_t threads, const int64_t* batch_subset,
                int64_t n_subset, double* phi, double* phi_abs, double* timings);

/* Algorithm 1 in parts: the setup (trees and modified charges) once, then evaluations of
 * all or some batches over it.  The input arrays must outlive the handle. */
typedef struct oracle_prepared oracle_prepared;
int oracle_bltc_prepare(const double* tx, const double* ty, const double* tz, int64_t nt,
                        const double* sx, const double* sy, const double* sz, const double* sq,
                        int64_t ns, double theta, int32_t degree, int32_t leaf_size,
                        int32_t batch_size, int32_t kernel, double kappa, int32_t threads,
                        oracle_prepared** out, double* timings);
int64_t oracle_bltc_num_batches(const oracle_prepared* p);
int oracle_bltc_evaluate(const oracle_prepared* p, const int64_t* batch_subset, int64_t n_subset,
                         int32_t threads, double* phi, double* phi_abs, double* seconds);
void oracle_bltc_release(oracle_prepared* p);

/* Algorithm 1 for distinct target and source sets (nt targets, ns sources). */
int oracle_bltc_ts(const double* tx, const double* ty, const double* tz, int64_t nt,
                   const double* sx, const double* sy, const double* sz, const double* sq,
                   int64_t ns, double theta, int32_t degree, int32_t leaf_size,
                   int32_t batch_size, int32_t kernel, double kappa, int32_t threads,
                   const int64_t* batch_subset, int64_t n_subset, double* phi, double* phi_abs,
                   double* timings);

/* Cluster-particle variant: targets clustered (leaf_size) and interpolated, sources in
 * batches (batch_size) summed exactly; the same MAC and exact-hit rules. */
int oracle_bltc_cp(const double* tx, const double* ty, const double* tz, int64_t nt,
                   const double* sx, const double* sy, const double* sz, const double* sq,
                   int64_t ns, double theta, int32_t degree, int32_t leaf_size,
                   int32_t batch_size, int32_t kernel, double kappa, int32_t threads,
                   double* phi, double* phi_abs);

/* Cluster-cluster variant (dual tree traversal): sources in a tree with leaf_size,
 * targets in a tree with batch_size; CC, CP, PC and PP interactions, then interpolation. */
int oracle_bltc_cc(const double* tx, const double* ty, const double* tz, int64_t nt,
                   const double* sx, const double* sy, const double* sz, const double* sq,
                   int64_t ns, double theta, int32_t degree, int32_t leaf_size,
                   int32_t batch_size, int32_t kernel, double kappa, int32_t threads,
                   double* phi, double* phi_abs);
/* The dual traversal's four lists (CC, CP, PC, PP) as (target node, source node) pairs;
 * counts[4]; t_ids/s_ids sized sum(counts) (NULL on a first call for the counts). */
int oracle_dual_lists_export(const oracle_tree* tt, const oracle_tree* st, double theta,
                             int32_t degree, int64_t* counts, int64_t* t_ids, int64_t* s_ids);

/* Barycentric Hermite treecode (future work of Sec. V; reading in bltc_oracle.c). */
void oracle_hermite_factors(int32_t degree, double lo, double hi, double y, double* h, double* k);
int oracle_kernel_dG(int32_t kernel, double kappa, int32_t kdeg, const double* x, const double* y,
                     double* out);
int oracle_hermite_charges(const oracle_tree* t, const double* x, const double* y, const double* z,
                           const double* q, int32_t degree, int32_t threads, double* qh);
int oracle_bltc_hermite(const double* x, const double* y, const double* z, const double* q, int64_t n,
                        double theta, int32_t degree, int32_t leaf_size, int32_t batch_size,
                        int32_t kernel, double kappa, int32_t threads, double* phi, double* phi_abs);

int oracle_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
