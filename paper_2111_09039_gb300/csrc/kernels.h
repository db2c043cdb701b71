// Launchers of the HSIM CUDA kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

struct __nv_bfloat16;

namespace hsim {
namespace k {

// ---- sparse (k_sparse.cu) -------------------------------------------------
// per-triangle cotangents and areas from positions or squared lengths
void triangle_geometry(cudaStream_t s, int m, const int *F, const double *V, const double *L2,
                       double *cot, double *area);
// S values in a CSR pattern: off-diagonal -1/2 sum of the opposite cotangents
// listed in ecot (two slots per entry, -1 = none), diagonal = -row sum;
// M diagonal = sum of incident areas / 3 (vertex -> triangle CSR vt_ptr/vt_idx),
// or with `consistent` the consistent mass in the same pattern
void assemble_sm(cudaStream_t s, int n, const int *ptr, const int *col, const int *ecot,
                 const double *cot, const int *vt_ptr, const int *vt_idx, const double *area,
                 double *S_val, double *M_diag, bool consistent);
// out[i] = sum of row i of a CSR matrix
void row_sums(cudaStream_t s, int n, const int *ptr, const double *val, double *out);
// dV = sum_i dloss[i] d lambda_i / dV (k_grad.cu); dV is zeroed first
void eig_grad(cudaStream_t s, int n, int m, int p, const double *V, const int *F, const double *evals,
              const double *evecs, int ld, const double *dloss, double *dV);
// Y[r, 0:k] = sum A[r,c] X[c, 0:k]
void spmm(cudaStream_t s, int n_rows, const int *ptr, const int *col, const double *val, int k,
          const double *X, int ldx, double *Y, int ldy);
// R = B - (S - mu M) X with M in S's pattern (M) or diagonal (Md)
void shifted_residual(cudaStream_t s, int n_rows, const int *ptr, const int *col, const double *S,
                      const double *M, const double *Md, double mu, int k, const double *X, int ldx,
                      const double *B, int ldb, double *R, int ldr);
// Y += X
void axpy_matrix(cudaStream_t s, int n, int k, const double *X, int ldx, double *Y, int ldy);
// Y[r, :] = d[r] * X[r, :]
void diag_scale(cudaStream_t s, int n, int k, const double *d, const double *X, int ldx, double *Y,
                int ldy);
// T = A U in a given pattern (rows of A)
void galerkin_au(cudaStream_t s, int n, const int *a_ptr, const int *a_col, const double *a_val,
                 const int *u_ptr, const int *u_col, const double *u_val, const int *t_ptr,
                 const int *t_col, double *t_val);
// C = U^T T in a given pattern; ut = transpose of U with values
void galerkin_utt(cudaStream_t s, int nc, const int *ut_ptr, const int *ut_col, const double *ut_val,
                  const int *t_ptr, const int *t_col, const double *t_val, const int *c_ptr,
                  const int *c_col, double *c_val);
// out[e] = in[map[e]]
void gather_values(cudaStream_t s, int64_t n, const int64_t *map, const double *in, double *out);
void gather_values_i(cudaStream_t s, int64_t n, const int *map, const double *in, double *out);
// Y[i, 0:k] = X[perm[i], 0:k]   (row gather)
void gather_rows(cudaStream_t s, int n, int k, const int *perm, const double *X, int ldx, double *Y,
                 int ldy);
// dense row-major n x n from CSR (zero elsewhere)
void densify(cudaStream_t s, int n, const int *ptr, const int *col, const double *val, double *D);
void densify_diag(cudaStream_t s, int n, const double *d, double *D);
// evecs column-major n x p (natural order) from Phi row-major internal
// (row iperm[i]); sign so that the entry of largest magnitude is positive
void output_evecs(cudaStream_t s, int n, int p, const int *iperm, const double *Phi, int ldp,
                  double *out, double *scratch_p);
void copy_matrix(cudaStream_t s, int rows, int cols, const double *X, int ldx, double *Y, int ldy);
// strided type conversions and FP32 helpers of the mixed-precision path
void convert_matrix(cudaStream_t s, int rows, int cols, const double *X, int ldx, float *Y, int ldy);
void convert_matrix(cudaStream_t s, int rows, int cols, const float *X, int ldx, double *Y, int ldy);
// R (FP32) = SP - rho MP column-wise, rho_j = num[j] / den[j] (den NULL: num[j]),
// formed once per column into rho (cols doubles of scratch); the difference
// in FP64, then truncated to FP32
void residual_f32(cudaStream_t s, int rows, int cols, const double *SP, int lds, const double *MP, int ldm,
                  const double *num, const double *den, double *rho, float *R, int ldr);
// the same with M = diag(m): R = SP - rho_j m_i X
void residual_f32_diag(cudaStream_t s, int rows, int cols, const double *SP, int lds, const double *X, int ldx,
                       const double *m, const double *num, const double *den, double *rho, float *R, int ldr);
// Y (FP64) = X - Z (FP32)
void sub_f2d(cudaStream_t s, int rows, int cols, const double *X, int ldx, const float *Z, int ldz, double *Y,
             int ldy);
void copy_matrix(cudaStream_t s, int rows, int cols, const float *X, int ldx, float *Y, int ldy);
void diag_scale(cudaStream_t s, int n, int k, const float *d, const float *X, int ldx, float *Y, int ldy);
// y = 1 / x
void reciprocal(cudaStream_t s, int n, const double *x, double *y);
void convert_f2d(cudaStream_t s, int64_t n, const float *x, double *y);
void convert_d2f(cudaStream_t s, int64_t n, const double *x, float *y);

// ---- dense (k_dense.cu) ---------------------------------------------------
// G (ka x kb, ld ldg, FP64) = A^T B over n rows; G is overwritten
template <typename T>
void gram(cudaStream_t s, int n, int ka, int kb, const T *A, int lda, const T *B, int ldb,
          double *G, int ldg, bool lower_only);
// C (n x m) = A (n x k) B (k x m), B in FP64
template <typename T>
void gemm_nn(cudaStream_t s, int n, int k, int m, const T *A, int lda, const double *B, int ldb,
             T *C, int ldc);
// residual sums: out[3j+0] = sum w R^2, +1 = sum w (S Phi)^2, +2 = sum w (M Phi)^2
// with R = SPhi - lam * MPhi; w = dinv (M^{-1}-norm) or 1 (2-norm)
template <typename T>
void residual_sums(cudaStream_t s, int n, int k, const T *SP, int lds, const T *MP, int ldm,
                   const double *lam, const double *dinv, double *out);
// w1 = diag(X^T Y1), w2 = diag(X^T Y2) (mixed path, FP32 products and sums
// per 256-row block, FP64 totals)
void col_dots2_mixed(cudaStream_t s, int n, int k, const double *X, int ldx, const double *Y1, const double *Y2,
                     int ldy, double *w1, double *w2);
// col_dots2_mixed with Y2 = diag(m) X (M not formed)
void col_dots2_diag_mixed(cudaStream_t s, int n, int k, const double *X, int ldx, const double *Y1, int ldy,
                          const double *m, double *w1, double *w2);
// residual_sums of the mixed path: the residual in FP64, the sums of squares
// accumulated in FP32 over 256-row blocks (relative accuracy ~1e-6)
void residual_sums_mixed(cudaStream_t s, int n, int k, const double *SP, int lds, const double *MP, int ldm,
                         const double *lam, const double *dinv, double *out);
// dense symmetric generalised eigensolver, k x k: LDL^T of M_bar, the lowest
// m (<= 0: all k) pairs of C^-1 S_bar C^-T by sym_eig, X (k x m) = C^-T V;
// returns 0 ok, 1 not SPD; *sweeps = 0 (kept for the Jacobi variant's report).
// tc: C^-1 formed explicitly and the transforms done as FP64-accurate
// tensor-core products (else FP64 triangular solves on the front kernels).
int ritz(cudaStream_t s, int k, const double *Sbar, int lds, const double *Mbar, int ldm, double *evals,
         double *X, int ldx, double *work, int *sweeps, int *flag_dev, int *flag_host, int m = 0, bool tc = false);
// ---- tridiagonal eigensolver (k_tridiag.cu) ----------------------------------
// lowest m eigenpairs of the symmetric n x n A (row-major, ld n, destroyed):
// evals ascending (m), X (n x m, ld ldx) orthonormal eigenvectors; work of
// sym_eig_work_size(n, m) doubles; synchronises the stream
size_t sym_eig_work_size(int n, int m);
void sym_eig(cudaStream_t s, int n, int m, double *A, double *evals, double *X, int ldx, double *work);
size_t ritz_work_size(int k);
// w = diag(M)^-1/2; S <- W S W, M <- W M W (q x q): unit-M-norm columns on the reduced side
void scale_sym_unit_diag(cudaStream_t s, int q, double *S, double *M, int lda, double *w);

// ---- fronts (k_front.cu) ----------------------------------------------------
struct FrontDev {
    const int64_t *foff;
    const int *nf, *ns, *pstart;
    const int64_t *rows_off;
    const int *rows;
    const int64_t *relmap_off;
    const int *relmap;
};
template <typename T>
void front_assemble(cudaStream_t s, int64_t nnz, const int *row_of, const int *col, const int64_t *dst,
                    const double *S_val, const double *M_val, const double *M_diag, double mu, T *arena);
template <typename T>
void front_extend_add(cudaStream_t s, const FrontDev &fd, const int *parent, const int *children,
                      int n_children, int max_upd, T *arena);
template <typename T>
void front_panel(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0,
                 int max_rows, T *arena, double pivot_tol, int *flags);
// c_end (front-local column): only the trailing columns below c_end are
// updated (the blocked factorisation's in-block updates); INT_MAX: all
template <typename T>
void front_update(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0,
                  int max_trail, T *arena, int c_end);
// max |F_t[i,i]| over the pivots of nodes 0..n_nodes-1 (bit pattern of a
// non-negative double, atomically maximised into *out)
template <typename T>
void front_maxdiag(cudaStream_t s, const FrontDev &fd, int n_nodes, const T *arena, unsigned long long *out);
template <typename T>
void front_diag(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, const T *arena,
                T *dpos, int *neg_count);
template <typename T>
void solve_fwd_tri(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0,
                   const T *arena, int k, T *X, int ldx);
template <typename T>
void solve_fwd_upd(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0,
                   int max_rows, const T *arena, int k, T *X, int ldx);
template <typename T>
void solve_diag(cudaStream_t s, int n, int k, const T *dpos, T *X, int ldx);
template <typename T>
void solve_bwd_upd(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0,
                   int max_rows, const T *arena, int k, T *X, int ldx);
template <typename T>
void solve_bwd_tri(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0,
                   const T *arena, int k, T *X, int ldx);
// fused forward / backward solve of single-panel fronts (ns <= kPanel,
// nf <= kSmallNf): triangle and update in one launch per tree height
constexpr int kSmallNf = 320;
template <typename T>
void solve_fwd_small(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int nf_max, const T *arena,
                     int k, T *X, int ldx);
template <typename T>
void solve_bwd_small(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int nf_max, const T *arena,
                     int k, T *X, int ldx);

// ---- inverted-factor solves (k_finv.cu) ------------------------------------
// One product of the front inversion, all operands column-major:
//   C = (+/-) A B,  A(i, k) = Abase[a + k lda + i],  B(k, j) = Bbase[b + j ldb + k],
//   C(i, j) = Cbase[c + j ldc + i],
// with A or B read as unit lower triangular (diagonal 1, upper part 0; the
// stored diagonal and upper part are not read) when flagged.  tile0 is the
// first 64 x 64 output tile of the task in the launch (prefix over tasks).
struct GemmTask {
    int64_t a, b, c;
    int M, N, K, lda, ldb, ldc, tile0, flags;
};
constexpr int kGemmAUnitLower = 1, kGemmBUnitLower = 2, kGemmNeg = 4;
constexpr int kGemmTile = 64;
// Tasks of the in-place inversion of the pivot blocks of fronts (nf[t] x
// nf[t] column-major at foff[t], ns[t] pivots): the 32 x 32 diagonal blocks;
// per block-doubling level bs = 32, 64, ... the products T = B Ainv (into
// scratch) and B <- -Cinv T for every pair of inverted diagonal blocks
// [a0, a0 + bs), [a0 + bs, a0 + 2 bs); then W = L_bs Linv (into scratch) and
// its copy over L_bs.  scratch: elements needed by the largest pass.
struct InversePlan {
    std::vector<int2> blk;
    std::vector<std::vector<GemmTask>> p1, p2;
    std::vector<int> tiles;
    std::vector<GemmTask> w, wc;
    int wtiles = 0;
    int64_t scratch = 0;
};
InversePlan inverse_plan(const std::vector<int> &nf, const std::vector<int> &ns, const std::vector<int64_t> &foff);

// The lowest two tree heights of the FP32 inverted-form solves in one launch
// each way (k_finv.cu): per listed front of height 1 (parents), its children
// child_ids[child_ptr[i] .. child_ptr[i + 1]) (leaves) and itself.  The
// forward stores D^-1 Y on these fronts' rows, which only the fused backward
// reads.  max_front bounds fused_front_size(nf, ns) of every front involved,
// max_rows nf + the children's pivots of every parent; parents have at most
// fused_max_pivots() pivots, fused_max_ancestors() rows beyond them and
// fused_max_children() children.  The results of solve_fwd_inv /
// solve_bwd_inv on heights 0 and 1 of those fronts, summed in another order.
constexpr size_t kFusedSmemMax = 160 * 1024;
// Shared memory of one fused CTA at most: three CTAs per SM
constexpr size_t kFuseSmemCap = 74 * 1024;
// The fused launches' plan (host): the fronts of height 1 within the fused
// kernels' limits (pivots, ancestor rows, children) whose CTA, sized for the
// largest front and rows of the launch, fits smem_cap (par, with children
// cid[cptr[i] .. cptr[i + 1]) in the order of h0), then the leaves (rest0)
// and fronts of height 1 (rest1) left to the per-height kernels; rows and
// front size the launch (max_rows and max_front of solve_fwd_fused).
struct FusePlan {
    std::vector<int> par, cptr, cid, rest0, rest1;
    int rows = 0, front = 0;
};
FusePlan fuse_plan(const std::vector<int> &nf, const std::vector<int> &ns, const std::vector<int> &parent,
                   const std::vector<int> &h0, const std::vector<int> &h1, size_t smem_cap);
size_t fused_smem(int max_rows, int max_front);
int fused_max_pivots();
int fused_max_ancestors();
int fused_max_children();
int fused_front_size(int nf, int ns);
void solve_fwd_fused(cudaStream_t s, const FrontDev &fd, const int *parents, int n_parents, const int *child_ptr,
                     const int *child_ids, int max_rows, int max_front, const float *arena, const float *dinv, int k,
                     float *X, float *Y, int ldx);
void solve_bwd_fused(cudaStream_t s, const FrontDev &fd, const int *parents, int n_parents, const int *child_ptr,
                     const int *child_ids, int max_rows, int max_front, const float *arena, int k, float *X,
                     const float *Y, int ldx);

// FP32-accurate products on the tcgen05 tensor cores (k_tc32.cu: operands
// split into two TF32 halves, three MMAs per K step, FP32 accumulators in
// TMEM; 128 x 128 output tiles).  The same operations as solve_fwd_inv and
// gemm_tasks for FP32 fronts.
void solve_fwd_tc(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int max_nf, const float *arena,
                  int k, float *X, float *Y, int ldx);
void gemm_tasks_tc(cudaStream_t s, const GemmTask *tasks, int ntasks, int tiles, const float *Ab, const float *Bb,
                   float *Cb);
// numbers the tasks' 128 x 128 tiles consecutively (tile0); returns the total
int gemm_tiles_tc(std::vector<GemmTask> &tasks);
// Schur-complement update of the blocked FP32 factorisation after a block of
// kSchurBlock pivot columns [K0, K0 + kSchurBlock): for every listed tile
// (node, m0, n0) of a front's trailing part (rows and columns from K0 +
// kSchurBlock on, lower triangle), F(r, c) -= sum_kk L(r, kk) d_kk L(c, kk)
// over the node's pivots kk of the block.
constexpr int kSchurBlock = 128;
struct SchurTask {
    int node, m0, n0;
};
void schur_tc(cudaStream_t s, const FrontDev &fd, const SchurTask *tasks, int ntasks, int K0, float *arena);
// fails with HSIM_E_TIMEOUT (and clears the flag) if a product's bounded
// mbarrier wait gave up since the last check
void tc32_check(cudaStream_t s);
// inverse of the unit lower 32 x 32 diagonal blocks (t, b0) of the pivot
// blocks, in place
template <typename T>
void inv_diag_blocks(cudaStream_t s, const FrontDev &fd, const int2 *blk, int nblk, T *arena);
template <typename T>
void gemm_tasks(cudaStream_t s, const GemmTask *tasks, int ntasks, int tiles, const T *Ab, const T *Bb, T *Cb);
// Cb[c + j ldc + i] = Ab[a + j lda + i], i < M, j < N, per task (64 x 64 tiles)
template <typename T>
void copy_tasks(cudaStream_t s, const GemmTask *tasks, int ntasks, int tiles, const T *Ab, T *Cb);
template <typename T>
void reciprocal(cudaStream_t s, int n, const T *x, T *y);
// forward substitution of one tree height on the inverted fronts:
// Y[pivots of t] = Linv_t X[pivots of t], X[ancestor rows of t] -= W_t X[pivots of t]
template <typename T>
void solve_fwd_inv(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int max_nf, int max_ns,
                   const T *arena, int k, T *X, T *Y, int ldx);
// backward substitution of one tree height: X[pivots of t] = Linv_t^T D^-1 Y[pivots of t] - W_t^T X[ancestor rows]
template <typename T>
void solve_bwd_inv(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int max_ns, const T *arena,
                   const T *dinv, int k, T *X, const T *Y, int ldx);

// ---- FP64-accurate products on BF16 tensor cores (k_ozaki.cu) --------------
constexpr int kOzakiSlices = 6;
// digit slices of an FP64 block in the tiled layout of k_ozaki.cu: rows
// padded to rows_p (multiple of 128), K to kp (multiple of 32), zero filled;
// one exponent per row; `digits` slices of 8 bits (6: 47 bits per value, the
// FP64-accurate form; 5: 39 bits)
struct OzakiOperand {
    int rows = 0, rows_p = 0, kp = 0, digits = kOzakiSlices;
    __nv_bfloat16 *slices = nullptr;
    int *exps = nullptr;
};
// bytes of scratch for splitting an n x cols block per column (K = n), or a
// rows x k block per row (K = k)
size_t ozaki_cols_scratch(int n, int cols);
size_t ozaki_rows_scratch(int rows, int k);
// split X (row-major, K = n rows) per column into a transposed operand
OzakiOperand ozaki_split_cols(cudaStream_t s, int n, int cols, const double *X, int ldx, void *scratch,
                              int digits = kOzakiSlices);
// split X (row-major rows x k, K = k) per row
OzakiOperand ozaki_split_rows(cudaStream_t s, int rows, int k, const double *X, int ldx, void *scratch,
                              int digits = kOzakiSlices);
// C (X.rows x Y.rows, FP64) = X Y^T over K = k_len (= X.kp); splits <= 0 chooses a
// split-K count (C accumulated with atomics), 1 stores directly; lower: C is
// symmetric, only tiles meeting the lower triangle run and the epilogue
// writes each value and its mirror image (X.rows == Y.rows)
void ozaki_product(cudaStream_t s, const OzakiOperand &X, const OzakiOperand &Y, int k_len, double *C, int ldc,
                   int splits, bool lower = false);
// fails (HSIM_E_INTERNAL) if a tensor-core product kernel gave up waiting on
// one of its barriers since the last check; synchronises the stream
void ozaki_check(cudaStream_t s);

}  // namespace k
}  // namespace hsim
