/*
 * hsim.h -- C ABI of the GB300 Hierarchical Subspace Iteration Method.
 *
 * Computes the p lowest eigenpairs of the generalised Laplace-Beltrami
 * problem  S Phi = lambda M Phi  (eq. eigenProb, Sec. 3.1) on a triangle mesh
 * with the Hierarchical Subspace Iteration Method (Alg. 3): a vertex
 * hierarchy with nested function spaces (Sec. 4.1, Alg. 2), a dense solve on
 * the coarsest level, then subspace iterations (Alg. 1) on every finer level
 * started from the prolonged coarse eigenbasis.
 *
 * Conventions shared by every call
 *   - Pointers named *_dev are CUDA device pointers on the device of the
 *     context; pointers named *_host are host pointers.  The caller owns
 *     every buffer it passes; the library owns the hierarchy, the
 *     factorisations and all workspace.  A device-pointer argument that the
 *     CUDA runtime classifies as plain (unregistered) host memory or as
 *     memory of another device is refused with HSIM_E_INVALID_ARG before any
 *     kernel runs; pinned and managed memory are accepted.  Sizes and
 *     indices inside device arrays are not checked.
 *   - All device work is issued on the context's stream.  A call returns
 *     after the stream has drained, unless its comment says otherwise.
 *   - Dense matrices are stored row-major unless stated: element (i, j) of
 *     an r x c matrix with leading dimension ld is at [i * ld + j].
 *   - Errors: a call returns HSIM_OK or an error status; the thread-local
 *     message is then available from hsim_last_error().  On error, outputs
 *     are undefined.  No C++ exception crosses this boundary.
 *   - Sparse matrices are CSR with int32 row pointers and column indices,
 *     sorted column indices per row, and double values.
 */
#ifndef HSIM_H
#define HSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HSIM_OK = 0,
    HSIM_E_INVALID_ARG = 1,    /* bad size, pointer or option */
    HSIM_E_NOMEM = 2,          /* host or device allocation failed */
    HSIM_E_CUDA = 3,           /* a CUDA call failed */
    HSIM_E_BREAKDOWN = 4,      /* tiny pivot in the LDL^T factorisation */
    HSIM_E_NOT_SPD = 5,        /* reduced mass matrix not positive definite */
    HSIM_E_NO_CONVERGENCE = 6, /* max_iters reached on some level */
    HSIM_E_TIMEOUT = 7,        /* a bounded device-side wait gave up */
    HSIM_E_INTERNAL = 8
} hsim_status;

enum { HSIM_FP64 = 0, HSIM_MIXED = 1 };

/* Boundary condition on surfaces with boundary (Sec. 5).  NATURAL: the cotan
 * S and lumped M of the open mesh as they are (Neumann).  DIRICHLET: the
 * boundary vertices (endpoints of edges that one triangle holds) are
 * eliminated; the level-0 unknowns are the interior vertices in increasing id
 * (hsim_hier_dofs) and the hierarchy is built over them (sampling chooses
 * interior vertices only, distances over the whole surface). */
enum { HSIM_BOUNDARY_NATURAL = 0, HSIM_BOUNDARY_DIRICHLET = 1 };

/* Mass matrix of the finest level (hsim_options.mass, read by
 * hsim_build_hierarchy).  LUMPED: M^0 diagonal, M_ii = sum of A_t / 3 over the
 * triangles of vertex i (the paper's experiments).  CONSISTENT: the exact
 * integral M_ij = int phi_i phi_j (A_t / 6 on the diagonal, A_t / 12 per
 * edge), a non-diagonal M in S's pattern (Sec. 7: HSIM handles generalised
 * problems with non-diagonal M unchanged).  With the consistent M the
 * M^-1-norms of the finest level's convergence test (eq. conv2) are bounded
 * through the lumped mass M_L (its row sums): every element satisfies
 * M_L / 4 <= M <= M_L, so ||x||_{M_L^-1} <= ||x||_{M^-1} <= 2 ||x||_{M_L^-1},
 * and the test uses twice the lumped-norm ratio, an upper bound of the exact
 * one (hsim_info.max_residual reports that bound). */
enum { HSIM_MASS_LUMPED = 0, HSIM_MASS_CONSISTENT = 1 };

/* Solver options.  Defaults (hsim_default_options) follow the paper:
 * sigma = 7 (Sec. 5, support region), alpha = 0.1 (Alg. 3 shift index
 * floor(alpha p)), two inverse iterations per Rayleigh-Ritz step and locking
 * at tolerance/10 (Sec. 4.2). */
typedef struct {
    int levels;          /* T >= 1; <= 0 selects 3, or 2 when p <= 200 (Sec. 5) */
    double sigma;        /* prolongation support: ~sigma centres per row (eq. radius) */
    double alpha;        /* shift index j = floor(alpha p) (Alg. 3) */
    int max_iters;       /* subspace iterations per level before HSIM_E_NO_CONVERGENCE */
    int inv_iters;       /* inverse iterations per Rayleigh-Ritz step (paper: 2) */
    double lock_factor;  /* lock a converged prefix below lock_factor * tol */
    int precision;       /* HSIM_FP64: every step in FP64, the paper's shift.
                            HSIM_MIXED: shift below the spectrum,
                            mu = -max(lambda_ref, 0.01 Lambda_{q-1}) (K positive
                            definite), FP32 factor in inverted form and FP32 solves
                            of the inverse iterations in correction form against
                            FP64 bases (hsim_shifted_solve_f32); Gram products,
                            basis update and the Ritz transforms on BF16 tensor
                            cores with FP64-accurate digit splitting
                            (hsim_gram_tc, hsim_ritz_tc; the Grams with 5 digits
                            per value at tol >= 1e-6); dense eigensolver and
                            residual vectors FP64 (sums of squares of the
                            convergence test accumulated in FP32 per row block) */
    int start_vertex;    /* first vertex of farthest-point sampling (Alg. 2) */
    int leaf_size;       /* nested-dissection leaf size (tuning, default 32) */
    int q;               /* subspace size; <= 0 selects max(ceil(1.5p), p+8) */
    int refine;          /* HSIM_FP64 only: FP64 residual refinement of the last
                            inverse iteration of each Rayleigh-Ritz step: 0 =
                            automatic (switched on for a level once its residual
                            stops decreasing), 1 = always, -1 = never */
    int boundary;        /* HSIM_BOUNDARY_NATURAL (default) or _DIRICHLET; read by
                            hsim_build_hierarchy, fixed for the hierarchy */
    int plain_sim;       /* 1: plain subspace iteration (Alg. 1 alone, the paper's
                            comparison without a hierarchy).  Read by
                            hsim_build_hierarchy (a single sparse level, no
                            sampling or prolongation); hsim_solve then starts from
                            the initialisation heuristic of Sec. 3.2 (diag(M),
                            unit vectors at the q - 2 smallest k_ii/m_ii, one
                            random column, hsim_random_column(seed)) with the
                            shift sim_shift.  FP64 only. */
    double sim_shift;    /* plain_sim: the shift mu of Alg. 1 */
    uint64_t seed;       /* plain_sim: seed of the random column */
    int mass;            /* HSIM_MASS_LUMPED (default) or HSIM_MASS_CONSISTENT; read by
                            hsim_build_hierarchy, fixed for the hierarchy (not with
                            plain_sim) */
    int hier_device;     /* hsim_build_hierarchy: 1 (default) computes the farthest-point
                            order and the prolongations U^tau on the context's GPU, 0 on
                            the host; both give the same order and the same U bit for
                            bit (Sec. 4.1) */
} hsim_options;

/* Per-solve report (host struct, optional). */
typedef struct {
    int levels;
    int sizes[8];          /* n^tau, tau = 0..levels-1 */
    int iters[8];          /* subspace iterations per level (index tau) */
    double shift[8];       /* mu per level */
    double max_residual;   /* eq. conv2 on the finest level, i < p */
    int64_t factor_nnz[8]; /* stored entries of L per level */
    double factor_flops[8];
    double ms_galerkin, ms_coarse, ms_prolong, ms_factor, ms_solve, ms_spmm,
           ms_gram, ms_ritz, ms_update, ms_residual, ms_total;
    int q;
    int ritz_calls;        /* Rayleigh-Ritz solves of size q on the SIM levels */
    int ritz_sweeps;       /* mixed path: Newton-Schulz steps of the reduced mass
                              matrices' inverse square roots, summed over those
                              solves (0 for a solve that factored M_bar) */
    int coarse_sweeps;     /* the same for the coarsest dense eigenproblem */
    double ms_tc_product;  /* HSIM_MIXED: tensor-core product kernels alone (part of
                              ms_gram and ms_update, which include the digit split) */
    double solve_flops;    /* triangular-solve flops, 4 nnz(L) per right-hand side */
} hsim_info;

typedef struct hsim_ctx hsim_ctx;
typedef struct hsim_hier hsim_hier;

void hsim_default_options(hsim_options *opts);

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The stream is
 * borrowed, not owned. */
hsim_status hsim_create(int device, void *cuda_stream, hsim_ctx **out);
void hsim_destroy(hsim_ctx *ctx);

/* Thread-local message of the last failed call on this thread. */
const char *hsim_last_error(void);

/* Number of compute kernels this library has launched since the process
 * started (all contexts). */
uint64_t hsim_kernel_launches(void);

/* --------------------------------------------------------------------------
 * Hierarchy (Sec. 4.1), run once per mesh:
 *   - level sizes n^{T-1} = max(ceil(1.5p), 1000) and geometric growth
 *     (eqs. nT-1, growthRate; growth rate read as the (T-1)-th root);
 *   - farthest-point sampling with shortest-path distances over the edge
 *     graph (Alg. 2), on the GPU (opts->hier_device = 1, the default: one
 *     thread-block cluster, several samples per relaxation where the
 *     straight-line bound proves them independent) or on the host;
 *   - prolongations U^tau (eqs. radius, basis and row normalisation), rows =
 *     level-tau vertices, columns = level-(tau+1) vertices, on the GPU (one
 *     truncated search per centre) or on the host; both devices give the
 *     same order and U bit for bit;
 *   - on the host: patterns of the Galerkin products S^tau = U^T S U
 *     (Alg. 3), a nested-dissection ordering (subtrees on worker threads)
 *     and the supernodal symbolic analysis of each level's shifted matrix
 *     S^tau - mu M^tau.
 * V_host (n x 3 positions) or L2_host (n_tris x 3 squared edge lengths, L2[t*3+k]
 * = edge opposite corner k of triangle t, for intrinsic meshes) must be
 * given; F_host is n_tris x 3 vertex indices.  Result uploaded to the device.
 * opts->boundary = HSIM_BOUNDARY_DIRICHLET builds the hierarchy over the
 * interior vertices (see the enum).  The host work uses up to
 * HSIM_HOST_THREADS threads (default: the hardware concurrency); the result
 * does not depend on the thread count.
 * Errors (HSIM_E_INVALID_ARG): vertex index out of range, a degenerate or
 * non-finite edge, a non-manifold edge, start_vertex out of range (or on a
 * Dirichlet boundary), q larger than the coarsest level, more than 8 levels,
 * a connected component without any coarse vertex.
 * ------------------------------------------------------------------------ */
hsim_status hsim_build_hierarchy(hsim_ctx *ctx, int n_verts, int n_tris, const double *V_host,
                                 const int32_t *F_host, const double *L2_host, int p,
                                 const hsim_options *opts, hsim_hier **out);
void hsim_hier_destroy(hsim_hier *hier);

/* Level sizes and the farthest-point order (mesh vertex ids of the first
 * n^1 samples) of a hierarchy.  sizes_host has room for 8; order_host may be
 * NULL or have room for sizes[1] entries. */
hsim_status hsim_hier_info(const hsim_hier *hier, int *levels, int *sizes_host,
                           int32_t *order_host);

/* Mesh vertex id of each level-0 unknown (sizes[0] entries, host): the
 * identity for the natural boundary condition, the interior vertices in
 * increasing id for a Dirichlet boundary.  Rows of S^0, M^0 and of the
 * eigenvectors follow this list. */
hsim_status hsim_hier_dofs(const hsim_hier *hier, int32_t *dofs_host);

/* The CSR pattern of S^0 that hsim_solve expects (rows in mesh order, every
 * mesh edge plus the diagonal; with a Dirichlet boundary the rows and columns
 * of the interior vertices only, renumbered as hsim_hier_dofs), as device
 * pointers owned by the hierarchy. */
hsim_status hsim_hier_pattern(const hsim_hier *hier, int *n, int64_t *nnz,
                              const int32_t **row_ptr_dev, const int32_t **col_dev);

/* Prolongation U^tau (natural orders: rows level-tau vertices, columns
 * level-(tau+1) vertices) copied to host arrays; call with NULL arrays to get
 * the sizes first. */
hsim_status hsim_hier_prolongation(const hsim_hier *hier, int tau, int *rows, int *cols,
                                   int64_t *nnz, int32_t *row_ptr_host, int32_t *col_host,
                                   double *val_host);

/* Cotan stiffness S^0 and mass M^0 on the device (Sec. 3.1,
 * eq. massStiffMatrices; S_ij = -1/2 (cot a_ij + cot b_ij), S_ii = -sum_j
 * S_ij), S written into the hierarchy's pattern.  M_diag_dev receives, for a
 * hierarchy built with mass = HSIM_MASS_LUMPED, the n diagonal entries
 * M_ii = sum of A_t/3 over incident triangles; with HSIM_MASS_CONSISTENT the
 * consistent mass in S's pattern (nnz values, A_t/6 on the diagonal and
 * A_t/12 per edge).  An edge that one triangle holds takes one cotangent.
 * With a Dirichlet boundary the matrices of the whole mesh are restricted to
 * the interior vertices (diagonals keep the boundary edges' weights).
 * Exactly one of V_dev (n x 3) and L2_dev (n_tris x 3) is non-NULL. */
hsim_status hsim_assemble(hsim_ctx *ctx, const hsim_hier *hier, const double *V_dev,
                          const double *L2_dev, double *S_val_dev, double *M_diag_dev);

/* HSIM (Alg. 3): the p lowest eigenpairs of S Phi = lambda M Phi.
 *   S_val_dev   values of S^0 in the hierarchy's pattern (hsim_hier_pattern)
 *   M_diag_dev  M^0 as hsim_assemble writes it: the lumped diagonal (n), or
 *               for a hierarchy with mass = HSIM_MASS_CONSISTENT its values in
 *               S's pattern (nnz)
 *   tol         relative residual tolerance of eq. conv2 (M^{-1}-norm)
 *   evals_dev   out: p eigenvalues, ascending
 *   evecs_dev   out: n x p, COLUMN-major (evecs[i + k n] = Phi_k(i)),
 *               M-orthonormal, entry of largest magnitude positive
 *   info        optional host report */
hsim_status hsim_solve(hsim_ctx *ctx, hsim_hier *hier, const double *S_val_dev,
                       const double *M_diag_dev, int p, double tol, const hsim_options *opts,
                       double *evals_dev, double *evecs_dev, hsim_info *info);

/* A batch of independent HSIM solves (one per mesh, each with its own
 * hierarchy), run concurrently: `streams` worker threads (<= 0: 8, at most
 * nmesh), each with its own CUDA stream on the context's device, take the
 * meshes largest first (level-0 size); every solve is the hsim_solve path.  The paper has no
 * batched form; many small meshes only fill the GPU when their solves
 * overlap.
 *   hiers, S_vals, M_diags, p, evals, evecs: nmesh entries each, as for
 *       hsim_solve (device pointers on the context's device; a hierarchy may
 *       appear once, since it holds its solve's workspace)
 *   opts       applied to every mesh (NULL: each hierarchy's options)
 *   infos      optional, nmesh host reports
 * Work already queued on the context's stream (e.g. the assembly of S, M)
 * completes before the batch starts; the call returns when every solve is
 * done.  On error the status of the first failing mesh is returned, its
 * index in hsim_last_error(); meshes not yet started are skipped and the
 * outputs of the others are undefined. */
hsim_status hsim_solve_batched(hsim_ctx *ctx, int nmesh, hsim_hier *const *hiers, const double *const *S_vals,
                               const double *const *M_diags, const int *p, double tol, const hsim_options *opts,
                               double *const *evals, double *const *evecs, hsim_info *infos, int streams);

/* Shape gradient of a loss of the eigenvalues (first-order perturbation of
 * S Phi = lambda M Phi for M-normalised eigenvectors, differentiated through
 * the cotan stiffness and lumped mass of Sec. 3.1, eq. massStiffMatrices):
 *     dV[v] = sum_{i<p} dloss_dlambda[i] * phi_i^T (dS/dx_v - lambda_i dM/dx_v) phi_i.
 * For the spectral loss sum_i (lambda_i - lambda*_i)^2 pass
 * dloss_dlambda[i] = 2 (lambda_i - lambda*_i).  Valid for simple
 * eigenvalues; inside a cluster of equal eigenvalues only a loss symmetric
 * in the cluster has a gradient.  The derivative is the one of the lumped
 * mass (eigenpairs of a hierarchy built with HSIM_MASS_CONSISTENT need the
 * consistent mass's derivative, which this entry does not form).
 *   V_dev          n x 3 positions (row-major)
 *   F_dev          n_tris x 3 vertex indices in [0, n); triangles of
 *                  positive area (the cotangents divide by it)
 *   evals_dev      p eigenvalues; evecs_dev n x p COLUMN-major, leading
 *                  dimension n (as hsim_solve writes them), M-orthonormal;
 *                  for a Dirichlet boundary the interior eigenvectors
 *                  scattered to the mesh vertices with zeros on the boundary
 *                  (S_II and M_II are restrictions of S and M, so the same
 *                  formula holds)
 *   dloss_dlambda_dev  p weights
 *   dV_dev         out: n x 3 row-major, overwritten
 * All device pointers on the context's device; the call returns after the
 * context's stream drained.  Indices are not range-checked on the device. */
hsim_status hsim_eig_grad(hsim_ctx *ctx, int n, int n_tris, const double *V_dev, const int32_t *F_dev,
                          int p, const double *evals_dev, const double *evecs_dev,
                          const double *dloss_dlambda_dev, double *dV_dev);

/* --------------------------------------------------------------------------
 * Step-level entry points: each runs one step of the hot path on caller
 * buffers, for parity tests and benchmarking of single kernels.
 * ------------------------------------------------------------------------ */

/* Y[r, 0:k] = sum_c A[r, c] X[c, 0:k]  (CSR SpMM; the products S Psi,
 * M Psi of Alg. 1 and the prolongation U Phi of Alg. 3).  X is n_cols x k with
 * leading dimension ldx, Y is n_rows x k with leading dimension ldy. */
hsim_status hsim_spmm(hsim_ctx *ctx, int n_rows, int n_cols, const int32_t *row_ptr_dev,
                      const int32_t *col_dev, const double *val_dev, int k, const double *X_dev,
                      int ldx, double *Y_dev, int ldy);
/* G = A^T B (k_a x k_b, row-major, ld k_b) for tall A (n x k_a, ld lda) and
 * B (n x k_b, ld ldb): the reduced matrices Psi^T S Psi, Psi^T M Psi of Alg. 1. */
hsim_status hsim_gram(hsim_ctx *ctx, int n, int k_a, int k_b, const double *A_dev, int lda,
                      const double *B_dev, int ldb, double *G_dev);

/* C = A B for A (n x k, ld lda) and small B (k x m, ld ldb), C (n x m, ld ldc):
 * the basis update Phi = Psi Phi_bar of Alg. 1. */
hsim_status hsim_gemm_update(hsim_ctx *ctx, int n, int k, int m, const double *A_dev, int lda,
                             const double *B_dev, int ldb, double *C_dev, int ldc);

/* The same two products evaluated on BF16 tensor cores with FP64 accuracy
 * (mixed-precision path): every FP64 operand is split against a power of two
 * per row or column into 6 integer digits of at most 8 bits, digit products
 * are accumulated exactly in FP32 over chunks of 128 and summed in FP64; the
 * result matches the FP64 product to about 2^-47 of the row/column maxima.
 * hsim_gram_tc takes `digits` = 6 (that accuracy) or 5 (2^-39, 15 digit
 * products instead of 21; the solve's Grams at tolerances >= 1e-6).
 * Arguments as hsim_gram and hsim_gemm_update (G is ka x kb, ld kb). */
hsim_status hsim_gram_tc(hsim_ctx *ctx, int n, int k_a, int k_b, const double *A_dev, int lda,
                         const double *B_dev, int ldb, double *G_dev, int digits);
hsim_status hsim_gemm_update_tc(hsim_ctx *ctx, int n, int k, int m, const double *A_dev, int lda,
                                const double *B_dev, int ldb, double *C_dev, int ldc);

/* Dense generalised symmetric eigenproblem S_bar X = M_bar X Lambda (Alg. 1,
 * dense eigenproblem step; also the coarsest level of Alg. 3): LDL^T of
 * M_bar = C C^T, Householder tridiagonalisation, multisection and inverse
 * iteration on A = C^-1 S_bar C^-T, back-transformation, all in FP64.  S_bar
 * and M_bar are k x k row-major (read only); evals (k) ascending; X (k x k,
 * row-major, column j = eigenvector j, X^T M_bar X = I).  Returns
 * HSIM_E_NOT_SPD if M_bar is not positive definite.  sweeps_out (host) may
 * be NULL (always 0).  Scratch is allocated per call. */
hsim_status hsim_ritz(hsim_ctx *ctx, int k, const double *Sbar_dev, const double *Mbar_dev,
                      double *evals_dev, double *X_dev, int *sweeps_out);
/* The same solve as done by the mixed-precision path.  When a Gershgorin
 * bound puts ||M_bar - I||_2 below 1/2 (the reduced mass matrices of the
 * solve after the first iteration of a level), W = M_bar^-1/2 comes from a
 * Newton-Schulz iteration and A = W S_bar W, X = W V; otherwise, or if that
 * iteration stalls above max|I - W^2 M_bar| = 1e-12, C^-1 is formed
 * explicitly (LDL^T of M_bar, in-place inversion of L by block doubling, FP64)
 * and A = (C^-1 S_bar) C^-T, X = C^-T V.  Every product is FP64-accurate on
 * BF16 tensor cores (as hsim_gram_tc).  sweeps_out: the Newton-Schulz steps
 * taken, 0 on the factorisation path.  Arguments and errors as hsim_ritz. */
hsim_status hsim_ritz_tc(hsim_ctx *ctx, int k, const double *Sbar_dev, const double *Mbar_dev,
                         double *evals_dev, double *X_dev, int *sweeps_out);

/* Galerkin restriction C = U^T A U of a level matrix (Alg. 3): A is n x n
 * CSR, U is n x nc CSR; C is returned in the CSR pattern computed on the
 * host by this call (row_ptr/col/val device buffers allocated by the library
 * and released with hsim_free). */
hsim_status hsim_galerkin(hsim_ctx *ctx, int n, int nc, const int32_t *A_ptr_host,
                          const int32_t *A_col_host, const double *A_val_dev,
                          const int32_t *U_ptr_host, const int32_t *U_col_host,
                          const double *U_val_dev, int64_t *nnz_out, int32_t **C_ptr_dev,
                          int32_t **C_col_dev, double **C_val_dev);
void hsim_free(void *dev_ptr);

/* Sparse symmetric indefinite factorisation K = S - mu M = P^T L D L^T P
 * (Alg. 1, factorisation step; Sec. 3.2 "Direct solver") and the solve
 * K X = B for k right-hand sides, on one level of a hierarchy: tau selects
 * the level's pattern and ordering.  S_val/M_val are values in the level's
 * natural-order pattern (tau = 0: hsim_hier_pattern and the diagonal M^0;
 * tau >= 1: the Galerkin pattern, M in the same pattern).  B is n x k
 * row-major in the level's natural vertex order; X overwrites B. */
hsim_status hsim_level_pattern(const hsim_hier *hier, int tau, int *n, int64_t *nnz,
                               int32_t *row_ptr_host, int32_t *col_host);
hsim_status hsim_shifted_solve(hsim_ctx *ctx, hsim_hier *hier, int tau, const double *S_val_dev,
                               const double *M_val_dev, double mu, int k, double *B_dev, int ldb,
                               int *negative_pivots);
/* The same solve as done by the mixed-precision path: the factorisation in
 * FP32 rewritten into the inverted form (pivot blocks inverted once, one
 * batched product per tree height and direction) and the solve in FP32; B
 * and X stay FP64 (converted at the boundary).  Meant for positive definite
 * K (mu below the spectrum), as the mixed path shifts; accuracy about the
 * condition of K times 2^-24.  Pivots below 1e-7 max|K_ii| fail with
 * HSIM_E_BREAKDOWN. */
hsim_status hsim_shifted_solve_f32(hsim_ctx *ctx, hsim_hier *hier, int tau, const double *S_val_dev,
                                   const double *M_val_dev, double mu, int k, double *B_dev, int ldb,
                                   int *negative_pivots);

/* Allocation-free variant of hsim_ritz, for callers that cannot let a
 * library allocate device memory (a framework that reserves the whole
 * device pool for its own allocator, a latency-bound loop that must not enter
 * the driver's allocator, a host that forbids allocations by plugins).  The
 * paper has no counterpart.  It is the same Rayleigh-Ritz reduction as
 * hsim_ritz (LDL^T of M_bar = C C^T, standard problem C^-1 S_bar C^-T,
 * X = C^-T V), but the standard problem is solved by a parallel cyclic FP64
 * Jacobi instead of the tridiagonal eigensolver: sweeps_out (host, may be
 * NULL) receives the number of Jacobi sweeps (hsim_ritz reports 0 there).
 * Eigenvalues agree with hsim_ritz to rounding; eigenvectors up to sign.
 * Fails with HSIM_E_NOT_SPD if M_bar is not positive definite and with
 * HSIM_E_NO_CONVERGENCE if the sweeps still rotate after 40 sweeps (outputs
 * then undefined).
 *
 * Its scratch is one fixed device array inside this library, sized for
 * k <= HSIM_RITZ_NOALLOC_MAX (about 3.2 MB on every device that loads the
 * library, kept until the process exits); larger k fails with
 * HSIM_E_INVALID_ARG.  No cudaMalloc or cudaFree is called.  The caller owns
 * the inputs Sbar_dev, Mbar_dev (k x k row-major, read only) and the outputs
 * evals_dev (k) and X_dev (k x k row-major), all on the current device; work
 * is issued on cuda_stream (a cudaStream_t, NULL = legacy default stream).
 * The call synchronizes that stream several times (after the factorisation
 * of M_bar and after every sweep, to read the rotation count) and returns
 * only after the stream has drained, so it cannot be captured into a CUDA
 * graph.  The first call on a device (made while it is current) looks up the
 * array's device address.  All calls share the array: calls that
 * overlap on the GPU (other streams or host threads) race and must be
 * serialised by the caller. */
#define HSIM_RITZ_NOALLOC_MAX 256
hsim_status hsim_ritz_noalloc(void *cuda_stream, int k, const double *Sbar_dev, const double *Mbar_dev,
                              double *evals_dev, double *X_dev, int *sweeps_out);

/* Host-only check of the ordering and symbolic analysis: factors the
 * natural-order symmetric CSR matrix (ptr/col/val, host) over the same front
 * structures and in the same order as the GPU kernels and solves K X = B for
 * nrhs right-hand sides (B, X: n x nrhs row-major, host).  Reports the number
 * of negative pivots (Sylvester inertia: eigenvalues below the shift) and the
 * stored entries of L.  Needs no GPU; the solver never uses it. */
hsim_status hsim_check_symbolic(int n, const int32_t *ptr, const int32_t *col, const double *val,
                                int leaf_size, int nrhs, const double *B, double *X,
                                int *negative_pivots, int64_t *nnz_L);
/* The same host replay for the inverted form of the mixed path's solves
 * (FP64 on the host): after the factorisation every pivot block is inverted
 * in place by the tasks of the GPU's inversion plan (32 x 32 diagonal blocks,
 * block doubling, W = L_bs Linv), then one product per front and direction
 * in the GPU's order of tree heights.  Arguments and results as
 * hsim_check_symbolic, and:
 *   fused_h01: nonzero replays tree heights 0 and 1 in the order of the GPU's
 *     fused launches (each planned front of height 1 with its leaves, its
 *     rows held apart, D^-1 Y stored by the forward); 0 per height.
 *   fused_counts (host, may be NULL): 3 ints, the fronts of height 1 that
 *     the plan fuses, the leaves and the fronts of height 1 it leaves to the
 *     per-height products (all 0 when fused_h01 is 0 or the tree has one
 *     height).
 * Needs no GPU. */
hsim_status hsim_check_inverted(int n, const int32_t *ptr, const int32_t *col, const double *val,
                                int leaf_size, int nrhs, const double *B, double *X,
                                int *negative_pivots, int64_t *nnz_L, int fused_h01,
                                int *fused_counts);
/* Host replay of the mesh part of hsim_build_hierarchy: the level sizes
 * (eqs. nT-1 and growthRate), the farthest-point order (Alg. 2) and the
 * prolongations U^tau (eq. basis, rows normalised to one), computed by the
 * host code that hsim_build_hierarchy runs before its device uploads.  Needs
 * no GPU; the solver never uses it.
 *   n_verts, n_tris, V_host, F_host, L2_host, p, opts: as hsim_build_hierarchy
 *     (opts NULL = defaults; levels, start_vertex, sigma, q and boundary are
 *     used).
 *   levels, sizes, U_nnz, nnz0 (host, required): T, n^0..n^{T-1} (room for
 *     8), the entries of U^0..U^{T-2} (room for 7) and of the level-0 pattern.
 *   dofs, order, U_ptr, U_col, U_val, ptr0, col0, src0 (host, each may be
 *     NULL, e.g. in a first call that learns the sizes): the mesh vertex of
 *     each level-0 unknown (n^0 entries, as hsim_hier_dofs), the first n^1
 *     vertices of farthest-point sampling (nothing when T = 1), then the CSR
 *     arrays of U^0, U^1, ... one after another: U_ptr holds n^tau + 1
 *     offsets per U^tau (local to that U^tau), U_col (coarse-level index) and
 *     U_val U_nnz[tau] entries each; last the level-0 pattern that
 *     hsim_hier_pattern returns (ptr0: n^0 + 1, col0: nnz0 entries) and for
 *     each of its entries the entry of the whole mesh's matrix that
 *     hsim_assemble takes its value from, as row * n_verts + col (src0).
 * Errors: HSIM_E_INVALID_ARG for a bad mesh or arguments (as
 * hsim_build_hierarchy, and when a connected component of the mesh holds no
 * coarse vertex); nothing is written then. */
/* The random column of plain SIM's initial basis (host): entry i is
 * 2 u_i - 1 with u_i the top 53 bits of the i-th SplitMix64 output (Steele,
 * Lea and Flood, 2014) from state `seed`, times 2^-53, for the level-0
 * unknown i (natural order).  Needs no GPU. */
void hsim_random_column(int n, uint64_t seed, double *out_host);

/* Host part of plain SIM's initial basis, as hsim_solve builds it for a
 * level of n unknowns whose elimination order is perm (perm[pos] = natural
 * index): unit_pos[c] (q - 2 entries) = row, in that order, of the unit
 * vector of column 1 + c (the q - 2 smallest sdiag[i]/mdiag[i], ascending,
 * the lower natural index first on ties); rand_int[pos] (n entries) =
 * hsim_random_column(seed) at natural index perm[pos].  Column 0 is
 * mdiag[perm[pos]].  Host arrays; needs no GPU; the solver never calls it. */
hsim_status hsim_check_plain_basis(int n, const double *sdiag, const double *mdiag, const int32_t *perm,
                                   int q, uint64_t seed, int32_t *unit_pos, double *rand_int);

hsim_status hsim_check_hierarchy(int n_verts, int n_tris, const double *V_host, const int32_t *F_host,
                                 const double *L2_host, int p, const hsim_options *opts, int *levels,
                                 int *sizes, int64_t *U_nnz, int64_t *nnz0, int32_t *dofs,
                                 int32_t *order, int32_t *U_ptr, int32_t *U_col, double *U_val,
                                 int32_t *ptr0, int32_t *col0, int64_t *src0);

#ifdef __cplusplus
}
#endif

#endif /* HSIM_H */
