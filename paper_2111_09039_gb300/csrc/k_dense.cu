// Dense FP64 kernels of the subspace iteration (Alg. 1):
//   gram        S_bar = Psi^T (S Psi), M_bar = Psi^T (M Psi)  (tall-skinny, split-K)
//   gemm_nn     Phi = Psi Phi_bar                                (basis update)
//   residual sums of eq. conv2 (FP64, and the mixed path's FP32-accumulated
//               form), Rayleigh quotients of the mixed correction step
//   ritz        S_bar Phi_bar = M_bar Phi_bar Lambda_bar: M_bar = L D L^T
//               (front kernels on one dense front), A = C^-1 S_bar C^-T with
//               C = L D^1/2, the lowest eigenpairs of A by the tridiagonal
//               eigensolver of k_tridiag.cu, Phi_bar = C^-T V, ascending.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>

#include "common.h"
#include "host.h"
#include "fpconv.h"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace hsim {
namespace k {

namespace {

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// SMs of the current device (queried per call: a process may drive GPUs of
// different sizes; the attribute query costs about a microsecond)
int sm_count() {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    return c > 0 ? c : 1;
}

constexpr int TB = 64;  // output tile
constexpr int TK = 16;  // k step

// G[i0:i0+64, j0:j0+64] += sum_{r in chunk} A[r, i] B[r, j]
template <typename T>
__global__ void __launch_bounds__(256) k_gram(int n, int ka, int kb, const T *__restrict__ A, int lda,
                                              const T *__restrict__ B, int ldb, double *__restrict__ G,
                                              int ldg, int rows_per_split, int lower_only) {
    const int ti = blockIdx.x, tj = blockIdx.y;
    if (lower_only && tj > ti) return;
    const int i0 = ti * TB, j0 = tj * TB;
    const int r_beg = blockIdx.z * rows_per_split;
    const int r_end = min(n, r_beg + rows_per_split);
    __shared__ T As[TK][TB];
    __shared__ T Bs[TK][TB];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4] = {};
    for (int r0 = r_beg; r0 < r_end; r0 += TK) {
        for (int idx = threadIdx.x; idx < TK * TB; idx += 256) {
            int c = idx & 63, rr = idx >> 6;
            int r = r0 + rr;
            As[rr][c] = (r < r_end && i0 + c < ka) ? A[(size_t)r * lda + i0 + c] : 0.0;
            Bs[rr][c] = (r < r_end && j0 + c < kb) ? B[(size_t)r * ldb + j0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < TK; ++rr) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[rr][ty + 16 * u];
                b[u] = Bs[rr][tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int i = i0 + ty + 16 * u;
        if (i >= ka) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int j = j0 + tx + 16 * v;
            if (j < kb && (!lower_only || j <= i)) atomicAdd(&G[(size_t)i * ldg + j], (double)acc[u][v]);
        }
    }
}

__global__ void k_mirror_lower(int k, double *__restrict__ G, int ldg) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)k * k) return;
    int i = (int)(idx / k), j = (int)(idx % k);
    if (j > i) G[(size_t)i * ldg + j] = G[(size_t)j * ldg + i];
}

// C[r0:r0+64, j0:j0+64] = A[r, :] B[:, j]
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_nn(int n, int kk, int m, const T *__restrict__ A, int lda,
                                                 const double *__restrict__ B, int ldb, T *__restrict__ C,
                                                 int ldc) {
    const int r0 = blockIdx.x * TB, j0 = blockIdx.y * TB;
    __shared__ T As[TK][TB + 1];
    __shared__ T Bs[TK][TB];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4] = {};
    for (int k0 = 0; k0 < kk; k0 += TK) {
        for (int idx = threadIdx.x; idx < TK * TB; idx += 256) {
            int c = idx % TK, r = idx / TK;  // A tile: 64 rows x 16 cols
            As[c][r] = (r0 + r < n && k0 + c < kk) ? A[(size_t)(r0 + r) * lda + k0 + c] : 0.0;
            int jj = idx & 63, kr = idx >> 6;  // B tile: 16 rows x 64 cols
            Bs[kr][jj] = (k0 + kr < kk && j0 + jj < m) ? (T)B[(size_t)(k0 + kr) * ldb + j0 + jj] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < TK; ++c) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[c][ty + 16 * u];
                b[u] = Bs[c][tx + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int r = r0 + ty + 16 * u;
        if (r >= n) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int j = j0 + tx + 16 * v;
            if (j < m) C[(size_t)r * ldc + j] = acc[u][v];
        }
    }
}

constexpr int kRowsPerBlock = 256;



template <typename T>
__global__ void k_residual_sums(int n, int k, const T *__restrict__ SP, int lds, const T *__restrict__ MP,
                                int ldm, const double *__restrict__ lam, const double *__restrict__ dinv,
                                double *__restrict__ out) {
    const int r_beg = blockIdx.x * kRowsPerBlock;
    const int r_end = min(n, r_beg + kRowsPerBlock);
    for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < k; j += gridDim.y * blockDim.x) {
        double l = lam[j];
        double a0 = 0.0, a1 = 0.0, a2 = 0.0;
        for (int r = r_beg; r < r_end; ++r) {
            double s = SP[(size_t)r * lds + j], m = MP[(size_t)r * ldm + j];
            double rr = s - l * m;
            double w = dinv ? dinv[r] : 1.0;
            a0 += w * rr * rr;
            a1 += w * s * s;
            a2 += w * m * m;
        }
        atomicAdd(&out[3 * j], a0);
        atomicAdd(&out[3 * j + 1], a1);
        atomicAdd(&out[3 * j + 2], a2);
    }
}

// Mixed path, the Rayleigh quotients of the correction step: w1 = diag(X^T Y1),
// w2 = diag(X^T Y2) in one pass over X, products and sums in FP32 over a
// block of rows (the correction form is exact for any quotient; an FP32
// accurate one keeps the corrections small).
__global__ void k_col_dots2_mixed(int n, int k, const double *__restrict__ X, int ldx, const double *__restrict__ Y1,
                                  const double *__restrict__ Y2, int ldy, double *__restrict__ w1,
                                  double *__restrict__ w2) {
    const int r_beg = blockIdx.x * kRowsPerBlock;
    const int r_end = min(n, r_beg + kRowsPerBlock);
    for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < k; j += gridDim.y * blockDim.x) {
        float a1 = 0.f, a2 = 0.f;
        for (int r = r_beg; r < r_end; ++r) {
            const float x = d2f_trunc(X[(size_t)r * ldx + j]);
            a1 = fmaf(x, d2f_trunc(Y1[(size_t)r * ldy + j]), a1);
            a2 = fmaf(x, d2f_trunc(Y2[(size_t)r * ldy + j]), a2);
        }
        atomicAdd(&w1[j], (double)a1);
        atomicAdd(&w2[j], (double)a2);
    }
}

// as k_col_dots2_mixed with Y2 = diag(m) X: w2 = sum m_i x_i^2
__global__ void k_col_dots2_diag_mixed(int n, int k, const double *__restrict__ X, int ldx,
                                       const double *__restrict__ Y1, int ldy, const double *__restrict__ m,
                                       double *__restrict__ w1, double *__restrict__ w2) {
    const int r_beg = blockIdx.x * kRowsPerBlock;
    const int r_end = min(n, r_beg + kRowsPerBlock);
    for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < k; j += gridDim.y * blockDim.x) {
        float a1 = 0.f, a2 = 0.f;
        for (int r = r_beg; r < r_end; ++r) {
            const float x = d2f_trunc(X[(size_t)r * ldx + j]);
            a1 = fmaf(x, d2f_trunc(Y1[(size_t)r * ldy + j]), a1);
            a2 = fmaf(d2f_trunc(m[r]) * x, x, a2);
        }
        atomicAdd(&w1[j], (double)a1);
        atomicAdd(&w2[j], (double)a2);
    }
}

// Mixed path: the residual s - lambda m in FP64 (it cancels), the three sums of
// squares (positive terms, well conditioned) in FP32 over a block of rows
// before the FP64 atomics: one FP64 instruction per element instead of seven.
__global__ void k_residual_sums_mixed(int n, int k, const double *__restrict__ SP, int lds,
                                      const double *__restrict__ MP, int ldm, const double *__restrict__ lam,
                                      const double *__restrict__ dinv, double *__restrict__ out) {
    const int r_beg = blockIdx.x * kRowsPerBlock;
    const int r_end = min(n, r_beg + kRowsPerBlock);
    for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < k; j += gridDim.y * blockDim.x) {
        const double l = lam[j];
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int r = r_beg; r < r_end; ++r) {
            const double sv = SP[(size_t)r * lds + j], mv = MP[(size_t)r * ldm + j];
            const float rr = d2f_trunc(fma(-l, mv, sv)), sf = d2f_trunc(sv), mf = d2f_trunc(mv);
            const float w = dinv ? d2f_trunc(dinv[r]) : 1.f;
            a0 = fmaf(w * rr, rr, a0);
            a1 = fmaf(w * sf, sf, a1);
            a2 = fmaf(w * mf, mf, a2);
        }
        atomicAdd(&out[3 * j], (double)a0);
        atomicAdd(&out[3 * j + 1], (double)a1);
        atomicAdd(&out[3 * j + 2], (double)a2);
    }
}

__global__ void k_transpose(int k, const double *__restrict__ X, int ldx, double *__restrict__ Y, int ldy) {
    __shared__ double t[32][33];
    int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int r = by + yy, c = bx + threadIdx.x;
        if (r < k && c < k) t[yy][threadIdx.x] = X[(size_t)r * ldx + c];
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int r = bx + yy, c = by + threadIdx.x;
        if (r < k && c < k) Y[(size_t)r * ldy + c] = t[threadIdx.x][yy];
    }
}

// X[i, :] *= f(d[i]):  mode 0: 1/sqrt(d), mode 1: sqrt(d)
__global__ void k_row_scale_sqrt(int k, const double *__restrict__ d, double *__restrict__ X, int ldx, int mode) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)k * k) return;
    int i = (int)(idx / k), j = (int)(idx % k);
    double s = mode == 0 ? rsqrt(d[i]) : sqrt(d[i]);
    X[(size_t)i * ldx + j] *= s;
}

__global__ void k_symmetrize(int k, double *__restrict__ A, int lda) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)k * k) return;
    int i = (int)(idx / k), j = (int)(idx % k);
    if (j <= i) return;
    double v = 0.5 * (A[(size_t)i * lda + j] + A[(size_t)j * lda + i]);
    A[(size_t)i * lda + j] = v;
    A[(size_t)j * lda + i] = v;
}

__global__ void k_identity(int k, double *__restrict__ V, int ldv) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)k * k) return;
    int i = (int)(idx / k), j = (int)(idx % k);
    V[(size_t)i * ldv + j] = (i == j) ? 1.0 : 0.0;
}

// ---- cyclic parallel Jacobi -------------------------------------------------
// Round-robin (circle) pairing of m (even) players over m - 1 rounds:
// player m-1 meets r; for t = 1..m/2-1, (r + t) meets (r - t) mod (m - 1).
__device__ __forceinline__ void pairing(int i, int r, int m, int &partner, int &pair_id, int &first) {
    const int mm = m - 1;
    if (i == mm) {
        partner = r;
        pair_id = 0;
        first = 0;
        return;
    }
    int d = i - r;
    d %= mm;
    if (d < 0) d += mm;
    if (d == 0) {
        partner = mm;
        pair_id = 0;
        first = 1;
        return;
    }
    if (d <= (m - 2) / 2) {
        pair_id = d;
        partner = ((r - d) % mm + mm) % mm;
        first = 1;
    } else {
        int t = mm - d;
        pair_id = t;
        partner = (r + t) % mm;
        first = 0;
    }
}

// column i of the rotation J restricted to i's pair: J[a][i] for a = first, second
__device__ __forceinline__ void jcol(int first, double c, double s, double &jf, double &js) {
    if (first) { jf = c; js = -s; }
    else { jf = s; js = c; }
}

__global__ void k_jacobi_sweep(int k, int m, double *A, double *A2, double *V, double *V2, double *cs, int lda,
                               double tol, double abs_tol, unsigned long long *rotations) {
    cg::grid_group grid = cg::this_grid();
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int npairs = m / 2;
    unsigned long long local_rot = 0;
    for (int r = 0; r < m - 1; ++r) {
        // rotations of this round
        for (int64_t pidx = tid; pidx < npairs; pidx += nthreads) {
            int p, q;
            if (pidx == 0) {
                p = r;
                q = m - 1;
            } else {
                p = (r + (int)pidx) % (m - 1);
                q = ((r - (int)pidx) % (m - 1) + (m - 1)) % (m - 1);
            }
            double c = 1.0, s = 0.0;
            if (p < k && q < k) {
                double app = A[(size_t)p * lda + p], aqq = A[(size_t)q * lda + q], apq = A[(size_t)p * lda + q];
                if (fabs(apq) > abs_tol && fabs(apq) > tol * sqrt(fabs(app) * fabs(aqq))) {
                    double theta = (aqq - app) / (2.0 * apq);
                    double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + hypot(theta, 1.0));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                    ++local_rot;
                }
            }
            cs[2 * pidx] = c;
            cs[2 * pidx + 1] = s;
        }
        grid.sync();
        // A2 = J^T A J,  V2 = V J
        for (int64_t idx = tid; idx < (int64_t)k * k; idx += nthreads) {
            int i = (int)(idx / k), j = (int)(idx % k);
            int pi_, idi, fi, pj_, idj, fj;
            pairing(i, r, m, pi_, idi, fi);
            pairing(j, r, m, pj_, idj, fj);
            double ci = cs[2 * idi], si = cs[2 * idi + 1], cj = cs[2 * idj], sj = cs[2 * idj + 1];
            // pair members of i: (ai0 = first, ai1 = second)
            int ai0 = fi ? i : pi_, ai1 = fi ? pi_ : i;
            int aj0 = fj ? j : pj_, aj1 = fj ? pj_ : j;
            double jif, jis, jjf, jjs;
            jcol(fi, ci, si, jif, jis);
            jcol(fj, cj, sj, jjf, jjs);
            if (ai1 >= k) { jif = (ai0 == i) ? 1.0 : 0.0; jis = 0.0; }
            if (ai0 >= k) { jif = 0.0; jis = (ai1 == i) ? 1.0 : 0.0; }
            if (aj1 >= k) { jjf = (aj0 == j) ? 1.0 : 0.0; jjs = 0.0; }
            if (aj0 >= k) { jjf = 0.0; jjs = (aj1 == j) ? 1.0 : 0.0; }
            double v = 0.0;
            if (ai0 < k) {
                double row0 = 0.0;
                if (aj0 < k) row0 += A[(size_t)ai0 * lda + aj0] * jjf;
                if (aj1 < k) row0 += A[(size_t)ai0 * lda + aj1] * jjs;
                v += jif * row0;
            }
            if (ai1 < k) {
                double row1 = 0.0;
                if (aj0 < k) row1 += A[(size_t)ai1 * lda + aj0] * jjf;
                if (aj1 < k) row1 += A[(size_t)ai1 * lda + aj1] * jjs;
                v += jis * row1;
            }
            A2[(size_t)i * lda + j] = v;
            double w = 0.0;
            if (aj0 < k) w += V[(size_t)i * lda + aj0] * jjf;
            if (aj1 < k) w += V[(size_t)i * lda + aj1] * jjs;
            V2[(size_t)i * lda + j] = w;
        }
        grid.sync();
        double *t = A; A = A2; A2 = t;
        t = V; V = V2; V2 = t;
    }
    if (local_rot) atomicAdd(rotations, local_rot);
}

// rank of each eigenvalue in ascending order (ties by index)
__global__ void k_rank(int k, const double *__restrict__ A, int lda, int *__restrict__ rank,
                       double *__restrict__ evals_sorted) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    double li = A[(size_t)i * lda + i];
    int r = 0;
    for (int j = 0; j < k; ++j) {
        double lj = A[(size_t)j * lda + j];
        r += (lj < li) || (lj == li && j < i);
    }
    rank[i] = r;
    evals_sorted[r] = li;
}

// Y[:, rank[j]] = X[:, j]
__global__ void k_permute_cols(int k, const int *__restrict__ rank, const double *__restrict__ X, int ldx,
                               double *__restrict__ Y, int ldy) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)k * k) return;
    int i = (int)(idx / k), j = (int)(idx % k);
    Y[(size_t)i * ldy + rank[j]] = X[(size_t)i * ldx + j];
}

// one dense front of size k (pivots 0..k-1), cached per size
struct DenseFront {
    DevBuf<int64_t> foff, rows_off, relmap_off;
    DevBuf<int> nf, ns, pstart, rows, relmap, node;
    FrontDev fd{};
    // in-place inversion of the unit lower factor (inverse_plan of one front)
    DevBuf<int2> blk;
    int nblk = 0;
    std::vector<DevBuf<GemmTask>> p1, p2;
    std::vector<int> ntask, tiles;
    int64_t scratch = 0;
};

DenseFront &dense_front(int k, cudaStream_t s) {
    static std::mutex mu;
    static std::map<int, std::unique_ptr<DenseFront>> cache;
    std::lock_guard<std::mutex> lock(mu);
    int dev = 0;
    cudaGetDevice(&dev);
    int key = dev * 1000000 + k;
    auto it = cache.find(key);
    if (it != cache.end()) return *it->second;
    auto d = std::make_unique<DenseFront>();
    d->foff.upload(std::vector<int64_t>{0, (int64_t)k * k}, s);
    d->rows_off.upload(std::vector<int64_t>{0, (int64_t)k}, s);
    d->relmap_off.upload(std::vector<int64_t>{0, 0}, s);
    d->nf.upload(std::vector<int>{k}, s);
    d->ns.upload(std::vector<int>{k}, s);
    d->pstart.upload(std::vector<int>{0}, s);
    std::vector<int> rows(k);
    for (int i = 0; i < k; ++i) rows[i] = i;
    d->rows.upload(rows, s);
    d->relmap.upload(std::vector<int>{0}, s);
    d->node.upload(std::vector<int>{0}, s);
    InversePlan P = inverse_plan({k}, {k}, {0});
    d->nblk = (int)P.blk.size();
    d->blk.upload(P.blk, s);
    for (size_t lv = 0; lv < P.p1.size(); ++lv) {
        d->ntask.push_back((int)P.p1[lv].size());
        d->p1.emplace_back();
        d->p1.back().upload(P.p1[lv], s);
        d->p2.emplace_back();
        d->p2.back().upload(P.p2[lv], s);
    }
    d->tiles = P.tiles;
    d->scratch = P.scratch;
    HSIM_CUDA(cudaStreamSynchronize(s));
    d->fd = FrontDev{d->foff.p, d->nf.p, d->ns.p, d->pstart.p, d->rows_off.p, d->rows.p, d->relmap_off.p, d->relmap.p};
    auto &ref = *d;
    cache[key] = std::move(d);
    return ref;
}

}  // namespace

template <typename T>
void gram(cudaStream_t s, int n, int ka, int kb, const T *A, int lda, const T *B, int ldb, double *G, int ldg,
          bool lower_only) {
    if (ldg == kb) {
        HSIM_CUDA(cudaMemsetAsync(G, 0, (size_t)ka * kb * sizeof(double), s));
    } else {
        HSIM_CUDA(cudaMemset2DAsync(G, (size_t)ldg * sizeof(double), 0, (size_t)kb * sizeof(double), ka, s));
    }
    if (n <= 0 || ka <= 0 || kb <= 0) return;
    int ti = cdiv(ka, TB), tj = cdiv(kb, TB);
    int64_t tiles = lower_only ? (int64_t)ti * (ti + 1) / 2 : (int64_t)ti * tj;
    int64_t want = std::max<int64_t>(1, (4LL * sm_count() + tiles - 1) / tiles);
    int64_t rows = std::max<int64_t>(256, (n + want - 1) / want);
    rows = (rows + TK - 1) / TK * TK;
    unsigned splits = cdiv(n, rows);
    dim3 g(ti, tj, splits);
    k_gram<T><<<g, 256, 0, s>>>(n, ka, kb, A, lda, B, ldb, G, ldg, (int)rows, lower_only ? 1 : 0);
    HSIM_LAUNCHED();
    if (lower_only) {
        k_mirror_lower<<<cdiv((int64_t)ka * ka, 256), 256, 0, s>>>(ka, G, ldg);
        HSIM_LAUNCHED();
    }
}

template <typename T>
void gemm_nn(cudaStream_t s, int n, int kk, int m, const T *A, int lda, const double *B, int ldb, T *C, int ldc) {
    if (n <= 0 || m <= 0) return;
    dim3 g(cdiv(n, TB), cdiv(m, TB));
    k_gemm_nn<T><<<g, 256, 0, s>>>(n, kk, m, A, lda, B, ldb, C, ldc);
    HSIM_LAUNCHED();
}



template <typename T>
void residual_sums(cudaStream_t s, int n, int k, const T *SP, int lds, const T *MP, int ldm, const double *lam,
                   const double *dinv, double *out) {
    HSIM_CUDA(cudaMemsetAsync(out, 0, (size_t)3 * k * sizeof(double), s));
    if (n <= 0 || k <= 0) return;
    dim3 g(cdiv(n, kRowsPerBlock), cdiv(k, 256));
    k_residual_sums<T><<<g, 256, 0, s>>>(n, k, SP, lds, MP, ldm, lam, dinv, out);
    HSIM_LAUNCHED();
}

void col_dots2_mixed(cudaStream_t s, int n, int k, const double *X, int ldx, const double *Y1, const double *Y2,
                     int ldy, double *w1, double *w2) {
    HSIM_CUDA(cudaMemsetAsync(w1, 0, (size_t)k * sizeof(double), s));
    HSIM_CUDA(cudaMemsetAsync(w2, 0, (size_t)k * sizeof(double), s));
    if (n <= 0 || k <= 0) return;
    dim3 g(cdiv(n, kRowsPerBlock), cdiv(k, 256));
    k_col_dots2_mixed<<<g, 256, 0, s>>>(n, k, X, ldx, Y1, Y2, ldy, w1, w2);
    HSIM_LAUNCHED();
}

void col_dots2_diag_mixed(cudaStream_t s, int n, int k, const double *X, int ldx, const double *Y1, int ldy,
                          const double *m, double *w1, double *w2) {
    HSIM_CUDA(cudaMemsetAsync(w1, 0, (size_t)k * sizeof(double), s));
    HSIM_CUDA(cudaMemsetAsync(w2, 0, (size_t)k * sizeof(double), s));
    if (n <= 0 || k <= 0) return;
    dim3 g(cdiv(n, kRowsPerBlock), cdiv(k, 256));
    k_col_dots2_diag_mixed<<<g, 256, 0, s>>>(n, k, X, ldx, Y1, ldy, m, w1, w2);
    HSIM_LAUNCHED();
}

void residual_sums_mixed(cudaStream_t s, int n, int k, const double *SP, int lds, const double *MP, int ldm,
                         const double *lam, const double *dinv, double *out) {
    HSIM_CUDA(cudaMemsetAsync(out, 0, (size_t)3 * k * sizeof(double), s));
    if (n <= 0 || k <= 0) return;
    dim3 g(cdiv(n, kRowsPerBlock), cdiv(k, 256));
    k_residual_sums_mixed<<<g, 256, 0, s>>>(n, k, SP, lds, MP, ldm, lam, dinv, out);
    HSIM_LAUNCHED();
}

#define HSIM_DENSE_INSTANTIATE(T)                                                                              \
    template void gram<T>(cudaStream_t, int, int, int, const T *, int, const T *, int, double *, int, bool);  \
    template void gemm_nn<T>(cudaStream_t, int, int, int, const T *, int, const double *, int, T *, int);    \
    template void residual_sums<T>(cudaStream_t, int, int, const T *, int, const T *, int, const double *,     \
                                   const double *, double *);

HSIM_DENSE_INSTANTIATE(float)
HSIM_DENSE_INSTANTIATE(double)

// w = diag(M)^-1/2, then S <- W S W and M <- W M W (q x q, ld lda)
__global__ void k_unit_diag_w(int q, const double *__restrict__ M, int lda, double *__restrict__ w) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < q) w[i] = 1.0 / sqrt(M[(size_t)i * lda + i]);
}
__global__ void k_scale_sym2(int q, double *__restrict__ S, double *__restrict__ M, int lda,
                             const double *__restrict__ w) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)q * q) return;
    int i = (int)(idx / q), j = (int)(idx % q);
    const double f = w[i] * w[j];
    S[(size_t)i * lda + j] *= f;
    M[(size_t)i * lda + j] *= f;
}

void scale_sym_unit_diag(cudaStream_t s, int q, double *S, double *M, int lda, double *w) {
    if (q <= 0) return;
    k_unit_diag_w<<<cdiv(q, 128), 128, 0, s>>>(q, M, lda, w);
    HSIM_LAUNCHED();
    k_scale_sym2<<<cdiv((int64_t)q * q, 256), 256, 0, s>>>(q, S, M, lda, w);
    HSIM_LAUNCHED();
}

size_t ritz_work_size(int k) {
    const size_t kk = (size_t)k * k;
    // F W T d | sym_eig work | tensor-core path: Cr Cc V, inversion scratch
    // (at most k^2), digit slices of two k x k operands
    const size_t oz = (ozaki_rows_scratch(k, k) + ozaki_cols_scratch(k, k) + 7) / 8;
    return 3 * kk + 2 * (size_t)k + 64 + sym_eig_work_size(k, k) + 4 * kk + oz + 48;
}

// Cr = D^-1/2 Linv (row-major) and Cc = Cr^T (row-major) from the inverted
// factor F (column-major: Linv strictly below the diagonal, unit diagonal)
__global__ void k_cinv(int k, const double *__restrict__ F, const double *__restrict__ d, double *__restrict__ Cr,
                       double *__restrict__ Cc) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)k * k) return;
    const int i = (int)(idx / k), j = (int)(idx % k);
    const double v = (i > j ? F[(size_t)j * k + i] : (i == j ? 1.0 : 0.0)) * rsqrt(d[i]);
    Cr[(size_t)i * k + j] = v;
    Cc[(size_t)j * k + i] = v;
}

// ---- Newton-Schulz inverse square root of a reduced mass matrix -------------
// Gershgorin bound max_i sum_j |M_ij - delta_ij| of ||M - I||_2 (one warp per
// row; non-negative doubles order like their bit patterns)
__global__ void k_gershgorin_dev(int k, const double *__restrict__ M, int ldm, unsigned long long *out) {
    const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x & 31;
    if (row >= k) return;
    double sum = 0.0;
    for (int j = lane; j < k; j += 32) sum += fabs(M[(size_t)row * ldm + j] - (j == row ? 1.0 : 0.0));
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(sum));
}

// T = (3 I - P) / 2 and max |I - P| (into out, as above)
__global__ void k_ns_step(int k, const double *__restrict__ P, double *__restrict__ T, unsigned long long *out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (idx < (int64_t)k * k) {
        const int i = (int)(idx / k), j = (int)(idx % k);
        const double id = i == j ? 1.0 : 0.0;
        e = fabs(id - P[idx]);
        T[idx] = 0.5 * (3.0 * id - P[idx]);
    }
    for (int o = 16; o > 0; o >>= 1) e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(e));
}

// X[i, 0:cols] *= 1/sqrt(d[i])
__global__ void k_rows_rsqrt(int rows, int cols, const double *__restrict__ d, double *__restrict__ X, int ldx) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)rows * cols) return;
    int i = (int)(idx / cols), j = (int)(idx % cols);
    X[(size_t)i * ldx + j] *= rsqrt(d[i]);
}

// C = A B for k x k row-major FP64 blocks as an FP64-accurate tensor-core product
static void tc_mm(cudaStream_t s, int k, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
                  unsigned char *oz) {
    OzakiOperand a = ozaki_split_rows(s, k, k, A, lda, oz);
    OzakiOperand b = ozaki_split_cols(s, k, k, B, ldb, oz + ozaki_rows_scratch(k, k));
    ozaki_product(s, a, b, a.kp, C, ldc, 0);
}

// Z = M_bar^-1/2 by the coupled Newton-Schulz iteration Y_0 = M_bar, Z_0 = I,
// T_j = (3 I - Z_j Y_j) / 2, Y_{j+1} = Y_j T_j, Z_{j+1} = T_j Z_j, which
// converges quadratically when ||M_bar - I||_2 < 1; products on the tensor
// cores.  Used when a Gershgorin bound puts ||M_bar - I||_2 below 1/2 (the
// columns are scaled to unit M-norm, so M_bar is near I once the basis is
// nearly M-orthonormal).  buf: four k x k scratch blocks.  Returns the block
// that holds Z, or nullptr if the bound fails or the iteration does not reach
// max|I - Z Y| < 1e-12 within 12 steps (the caller then factors M_bar); the
// products carry about 2^-47 of their row and column maxima per term, so the
// attainable level near I is a few 1e-14 times sqrt(k).  *steps: iterations.
static const double *ns_inv_sqrt(cudaStream_t s, int k, const double *Mbar, int ldm, double *const buf[4],
                                 unsigned char *oz, unsigned long long *dmax, int *steps) {
    auto read_max = [&](double &v) {
        unsigned long long h = 0;
        HSIM_CUDA(cudaMemcpyAsync(&h, dmax, sizeof(h), cudaMemcpyDeviceToHost, s));
        HSIM_CUDA(cudaStreamSynchronize(s));
        std::memcpy(&v, &h, sizeof(v));
    };
    HSIM_CUDA(cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), s));
    k_gershgorin_dev<<<cdiv(k, 8), 256, 0, s>>>(k, Mbar, ldm, dmax);
    HSIM_LAUNCHED();
    double g = 1.0;
    read_max(g);
    if (!(g < 0.5)) return nullptr;
    double *Y = buf[0], *Z = buf[1], *P = buf[2], *T = buf[3];
    copy_matrix(s, k, k, Mbar, ldm, Y, k);
    k_identity<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, Z, k);
    HSIM_LAUNCHED();
    double prev = 1.0;
    for (int it = 0; it < 12; ++it) {
        tc_mm(s, k, Z, k, Y, k, P, k, oz);  // P = Z Y
        HSIM_CUDA(cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), s));
        k_ns_step<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, P, T, dmax);
        HSIM_LAUNCHED();
        double e = 1.0;
        read_max(e);
        if (e < 1e-12) {
            k_symmetrize<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, Z, k);
            HSIM_LAUNCHED();
            *steps = it;
            return Z;
        }
        if (!(e < 0.5 * prev) && it > 1) return nullptr;  // stopped contracting above the target
        prev = e;
        tc_mm(s, k, Y, k, T, k, P, k, oz);  // Y T
        std::swap(Y, P);
        tc_mm(s, k, T, k, Z, k, P, k, oz);  // T Z
        std::swap(Z, P);
    }
    return nullptr;
}

int ritz(cudaStream_t s, int k, const double *Sbar, int lds, const double *Mbar, int ldm, double *evals, double *X,
         int ldx, double *work, int *sweeps, int *flag_dev, int *flag_host, int m, bool tc) {
    // work layout: F (k*k) | W (k*k) | T (k*k) | d (k) | eigensolver work
    if (m <= 0 || m > k) m = k;
    const size_t kk = (size_t)k * k;
    double *F = work, *W = work + kk, *T = work + 2 * kk;
    double *d = T + kk;
    double *ework = d + 2 * (size_t)k + 32;
    DenseFront &df = dense_front(k, s);
    const int *node = df.node.p;
    if (tc) {
        // M_bar near I: W = M_bar^-1/2 by Newton-Schulz on the tensor cores
        // (W M_bar W = I), A = W S_bar W, X = W V; no factorisation of M_bar
        double *Cr = ework + sym_eig_work_size(k, k) + 8, *Cc = Cr + kk, *V = Cc + kk, *scr = V + kk;
        unsigned char *oz = reinterpret_cast<unsigned char *>(
            (reinterpret_cast<uintptr_t>(scr + kk) + 255) & ~static_cast<uintptr_t>(255));
        double *const buf[4] = {F, Cr, Cc, scr};
        int ns_steps = 0;
        const double *Wz =
            ns_inv_sqrt(s, k, Mbar, ldm, buf, oz, reinterpret_cast<unsigned long long *>(flag_dev + 4), &ns_steps);
        if (Wz) {
            if (sweeps) *sweeps = ns_steps;
            tc_mm(s, k, Wz, k, Sbar, lds, W, k, oz);
            tc_mm(s, k, W, k, Wz, k, T, k, oz);
            k_symmetrize<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, T, k);
            HSIM_LAUNCHED();
            sym_eig(s, k, m, T, evals, V, m, ework);
            OzakiOperand a = ozaki_split_rows(s, k, k, Wz, k, oz);
            OzakiOperand b = ozaki_split_cols(s, k, m, V, m, oz + ozaki_rows_scratch(k, k));
            ozaki_product(s, a, b, a.kp, X, ldx, 0);
            ozaki_check(s);
            return 0;
        }
    }
    // F = M_bar (symmetric: row-major == column-major); M_bar = L D L^T = C C^T
    copy_matrix(s, k, k, Mbar, ldm, F, k);
    HSIM_CUDA(cudaMemsetAsync(flag_dev, 0, 4 * sizeof(int), s));
    const int steps = (k + kPanel - 1) / kPanel;
    for (int st = 0; st < steps; ++st) {
        int k0 = st * kPanel;
        int kb = std::min(kPanel, k - k0);
        front_panel(s, df.fd, node, 1, k0, k - k0 - kb, F, 1e-300, flag_dev);
        front_update(s, df.fd, node, 1, k0, k - k0 - kb, F, INT_MAX);
    }
    front_diag(s, df.fd, node, 1, F, d, flag_dev + 2);
    HSIM_CUDA(cudaMemcpyAsync(flag_host, flag_dev, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaStreamSynchronize(s));
    if (flag_host[0] != 0 || flag_host[2] != 0) return 1;  // not positive definite
    if (sweeps) *sweeps = 0;
    if (tc) {
        // Cinv = D^-1/2 L^-1 explicitly (L inverted in place by block
        // doubling), then the three transforms as FP64-accurate tensor-core
        // products: A = (Cinv S_bar) Cinv^T, X = Cinv^T V
        const size_t kk = (size_t)k * k;
        double *Cr = ework + sym_eig_work_size(k, k) + 8, *Cc = Cr + kk, *V = Cc + kk, *scr = V + kk;
        // digit slices are read by bulk copies: 256-byte aligned base
        unsigned char *oz = reinterpret_cast<unsigned char *>(
            (reinterpret_cast<uintptr_t>(scr + kk) + 255) & ~static_cast<uintptr_t>(255));
        const size_t rb = ozaki_rows_scratch(k, k);
        HSIM_CHECK_ARG(df.scratch <= (int64_t)kk, "ritz: inversion scratch");
        inv_diag_blocks<double>(s, df.fd, df.blk.p, df.nblk, F);
        for (size_t lv = 0; lv < df.p1.size(); ++lv) {
            gemm_tasks<double>(s, df.p1[lv].p, df.ntask[lv], df.tiles[lv], F, F, scr);
            gemm_tasks<double>(s, df.p2[lv].p, df.ntask[lv], df.tiles[lv], F, scr, F);
        }
        k_cinv<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, F, d, Cr, Cc);
        HSIM_LAUNCHED();
        OzakiOperand a = ozaki_split_rows(s, k, k, Cr, k, oz);
        OzakiOperand b = ozaki_split_cols(s, k, k, Sbar, lds, oz + rb);
        ozaki_product(s, a, b, a.kp, W, k, 0);
        a = ozaki_split_rows(s, k, k, W, k, oz);
        b = ozaki_split_cols(s, k, k, Cc, k, oz + rb);
        ozaki_product(s, a, b, a.kp, T, k, 0);
        k_symmetrize<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, T, k);
        HSIM_LAUNCHED();
        sym_eig(s, k, m, T, evals, V, m, ework);
        a = ozaki_split_rows(s, k, k, Cc, k, oz);
        b = ozaki_split_cols(s, k, m, V, m, oz + rb);
        ozaki_product(s, a, b, a.kp, X, ldx, 0);
        ozaki_check(s);
        return 0;
    }
    // A = C^-1 S_bar C^-T: W = D^-1/2 L^-1 S_bar, T = D^-1/2 L^-1 W^T
    copy_matrix(s, k, k, Sbar, lds, W, k);
    auto forward = [&](double *Y) {
        for (int st = 0; st < steps; ++st) {
            int k0 = st * kPanel;
            int kb = std::min(kPanel, k - k0);
            solve_fwd_tri(s, df.fd, node, 1, k0, F, k, Y, k);
            solve_fwd_upd(s, df.fd, node, 1, k0, k - k0 - kb, F, k, Y, k);
        }
        k_row_scale_sqrt<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, d, Y, k, 0);
        HSIM_LAUNCHED();
    };
    forward(W);
    dim3 tg(cdiv(k, 32), cdiv(k, 32)), tb(32, 8);
    k_transpose<<<tg, tb, 0, s>>>(k, W, k, T, k);
    HSIM_LAUNCHED();
    forward(T);
    // symmetrise against rounding: T = (T + T^T)/2
    k_symmetrize<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, T, k);
    HSIM_LAUNCHED();
    // lowest m eigenpairs of A (ascending), eigenvectors into X (k x m)
    sym_eig(s, k, m, T, evals, X, ldx, ework);
    // X = C^-T V = L^-T D^-1/2 V
    k_rows_rsqrt<<<cdiv((int64_t)k * m, 256), 256, 0, s>>>(k, m, d, X, ldx);
    HSIM_LAUNCHED();
    for (int st = steps - 1; st >= 0; --st) {
        int k0 = st * kPanel;
        int kb = std::min(kPanel, k - k0);
        solve_bwd_upd(s, df.fd, node, 1, k0, k - k0 - kb, F, m, X, ldx);
        solve_bwd_tri(s, df.fd, node, 1, k0, F, m, X, ldx);
    }
    return 0;
}

// ===========================================================================
// Allocation-free Ritz solve.
//
// Some callers cannot let a library allocate device memory: a framework that
// reserves the whole device pool for its own caching allocator (a cudaMalloc
// from inside would fail or fragment it), a latency-bound loop that must not
// enter the driver's allocator, or a host that forbids allocations by plugins.
// For them hsim_ritz_noalloc runs the same Rayleigh-Ritz reduction as
// hsim_ritz (LDL^T of M_bar = C C^T, then the standard problem
// C^-1 S_bar C^-T), solved by a parallel cyclic FP64 Jacobi rather than the
// tridiagonal eigensolver of hsim_ritz, with all of its scratch taken from
// one fixed, file-scope device array (about 3.2 MB per device that loads the
// library, held until the process exits).  Its address
// is looked up once per device with cudaGetSymbolAddress, by the first call
// made while that device is current; that first call should therefore come
// before any stream capture.  Every call shares the array: calls whose work
// overlaps on the GPU (different streams, or different host threads) race and
// must be serialised by the caller.  The flags and counters that must start
// at zero are cleared by every call; everything else is overwritten before it
// is read.
// ===========================================================================
namespace {

constexpr int kNoAllocMaxK = HSIM_RITZ_NOALLOC_MAX;
constexpr int kMaxJacobiSweeps = 40;
constexpr size_t kNoAllocWork = (size_t)6 * kNoAllocMaxK * kNoAllocMaxK + 4 * (size_t)kNoAllocMaxK + 64;
// byte offsets inside the scratch array
constexpr size_t kOffWork = 0;
constexpr size_t kOffI64 = kOffWork + kNoAllocWork * sizeof(double);     // foff[2], rows_off[2], relmap_off[2]
constexpr size_t kOffI32 = kOffI64 + 6 * sizeof(int64_t);                // nf, ns, pstart, relmap, node, flags[4]
constexpr size_t kOffRows = kOffI32 + 16 * sizeof(int);                  // rows[kNoAllocMaxK]
constexpr size_t kNoAllocBytes = kOffRows + (size_t)kNoAllocMaxK * sizeof(int);

static __device__ __align__(256) unsigned char g_ritz_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_addr[kMaxDevices] = {};

// Device address of g_ritz_scratch for the current device (looked up once).
unsigned char *noalloc_scratch(int dev) {
    HSIM_CHECK_ARG(dev >= 0 && dev < kMaxDevices, "device index beyond the supported range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        HSIM_CUDA(cudaGetSymbolAddress(&ptr, g_ritz_scratch));
        g_noalloc_addr[dev] = static_cast<unsigned char *>(ptr);
    }
    return g_noalloc_addr[dev];
}

__global__ void k_noalloc_front(int k, int64_t *i64, int *i32, int *rows) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) rows[i] = i;
    if (i == 0) {
        i64[0] = 0;                 // foff
        i64[1] = (int64_t)k * k;
        i64[2] = 0;                 // rows_off
        i64[3] = k;
        i64[4] = 0;                 // relmap_off
        i64[5] = 0;
        i32[0] = k;                 // nf
        i32[1] = k;                 // ns
        i32[2] = 0;                 // pstart
        i32[3] = 0;                 // relmap
        i32[4] = 0;                 // node list
    }
}

// The Rayleigh-Ritz solve with the dense front description and the work area
// supplied by the caller: LDL^T of M_bar on the front kernels, the two
// triangular transforms, then cyclic Jacobi sweeps until a sweep applies no
// rotation.  Returns 0 on success, 1 if M_bar is not positive definite, 2 if
// the Jacobi sweeps still rotated after kMaxJacobiSweeps sweeps (the
// spectrum is then not converged and the vectors not M-orthonormal).
int ritz_on(cudaStream_t s, int k, const double *Sbar, int lds, const double *Mbar, int ldm, double *evals, double *X,
            int ldx, double *work, const FrontDev &fd, const int *node, int *sweeps, int *flag_dev, int *flag_host) {
    const size_t kk = (size_t)k * k;
    double *F = work, *A = work + kk, *A2 = work + 2 * kk, *V = work + 3 * kk, *V2 = work + 4 * kk, *W = work + 5 * kk;
    double *d = work + 6 * kk;
    double *cs = d + k;
    unsigned long long *rot = reinterpret_cast<unsigned long long *>(cs + k + 2);
    copy_matrix(s, k, k, Mbar, ldm, F, k);
    HSIM_CUDA(cudaMemsetAsync(flag_dev, 0, 4 * sizeof(int), s));
    const int steps = (k + kPanel - 1) / kPanel;
    for (int st = 0; st < steps; ++st) {
        int k0 = st * kPanel;
        int kb = std::min(kPanel, k - k0);
        front_panel(s, fd, node, 1, k0, k - k0 - kb, F, 1e-300, flag_dev);
        front_update(s, fd, node, 1, k0, k - k0 - kb, F, INT_MAX);
    }
    front_diag(s, fd, node, 1, F, d, flag_dev + 2);
    HSIM_CUDA(cudaMemcpyAsync(flag_host, flag_dev, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaStreamSynchronize(s));
    if (flag_host[0] != 0 || flag_host[2] != 0) return 1;
    copy_matrix(s, k, k, Sbar, lds, W, k);
    auto forward = [&](double *Y) {
        for (int st = 0; st < steps; ++st) {
            int k0 = st * kPanel;
            int kb = std::min(kPanel, k - k0);
            solve_fwd_tri(s, fd, node, 1, k0, F, k, Y, k);
            solve_fwd_upd(s, fd, node, 1, k0, k - k0 - kb, F, k, Y, k);
        }
        k_row_scale_sqrt<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, d, Y, k, 0);
        HSIM_LAUNCHED();
    };
    forward(W);
    dim3 tg(cdiv(k, 32), cdiv(k, 32)), tb(32, 8);
    k_transpose<<<tg, tb, 0, s>>>(k, W, k, A, k);
    HSIM_LAUNCHED();
    forward(A);
    k_symmetrize<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, A, k);
    HSIM_LAUNCHED();
    k_identity<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, V, k);
    HSIM_LAUNCHED();
    const int m = (k % 2) ? k + 1 : k;
    int blocks_per_sm = 0;
    HSIM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_jacobi_sweep, 256, 0));
    int grid = std::max(1, std::min(blocks_per_sm, 4) * sm_count());
    int64_t need = std::max<int64_t>((int64_t)k * k, m / 2);
    grid = (int)std::min<int64_t>(grid, (need + 255) / 256);
    grid = std::max(grid, 1);
    double tol = 1e-15, abs_tol = 1e-300;
    int sw = 0;
    unsigned long long hrot = 1;
    double *pA = A, *pA2 = A2, *pV = V, *pV2 = V2;
    while (hrot != 0 && sw < kMaxJacobiSweeps) {
        HSIM_CUDA(cudaMemsetAsync(rot, 0, sizeof(unsigned long long), s));
        int kk_ = k, mm = m, ld = k;
        void *args[] = {&kk_, &mm, &pA, &pA2, &pV, &pV2, &cs, &ld, &tol, &abs_tol, &rot};
        HSIM_CUDA(cudaLaunchCooperativeKernel((void *)k_jacobi_sweep, dim3(grid), dim3(256), args, 0, s));
        HSIM_LAUNCHED();
        if ((m - 1) % 2 == 1) {
            std::swap(pA, pA2);
            std::swap(pV, pV2);
        }
        HSIM_CUDA(cudaMemcpyAsync(&hrot, rot, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        HSIM_CUDA(cudaStreamSynchronize(s));
        ++sw;
    }
    if (sweeps) *sweeps = sw;
    if (hrot != 0) return 2;
    int *rk = reinterpret_cast<int *>(W);
    k_rank<<<cdiv(k, 128), 128, 0, s>>>(k, pA, k, rk, evals);
    HSIM_LAUNCHED();
    k_row_scale_sqrt<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, d, pV, k, 0);
    HSIM_LAUNCHED();
    for (int st = steps - 1; st >= 0; --st) {
        int k0 = st * kPanel;
        int kb = std::min(kPanel, k - k0);
        solve_bwd_upd(s, fd, node, 1, k0, k - k0 - kb, F, k, pV, k);
        solve_bwd_tri(s, fd, node, 1, k0, F, k, pV, k);
    }
    k_permute_cols<<<cdiv((int64_t)k * k, 256), 256, 0, s>>>(k, rk, pV, k, X, ldx);
    HSIM_LAUNCHED();
    return 0;
}

}  // namespace
}  // namespace k
}  // namespace hsim

extern "C" hsim_status hsim_ritz_noalloc(void *cuda_stream, int k, const double *Sbar_dev, const double *Mbar_dev,
                                         double *evals_dev, double *X_dev, int *sweeps_out) {
    using namespace hsim;
    try {
        HSIM_CHECK_ARG(Sbar_dev && Mbar_dev && evals_dev && X_dev, "NULL argument");
        HSIM_CHECK_ARG(k >= 1, "k must be >= 1");
        if (k > k::kNoAllocMaxK)
            fail(HSIM_E_INVALID_ARG, "hsim_ritz_noalloc: k = " + std::to_string(k) + " exceeds the fixed scratch limit " +
                                         std::to_string(k::kNoAllocMaxK) + "; use hsim_ritz");
        int dev = 0;
        HSIM_CUDA(cudaGetDevice(&dev));
        cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
        unsigned char *base = k::noalloc_scratch(dev);
        double *work = reinterpret_cast<double *>(base + k::kOffWork);
        int64_t *i64 = reinterpret_cast<int64_t *>(base + k::kOffI64);
        int *i32 = reinterpret_cast<int *>(base + k::kOffI32);
        int *rows = reinterpret_cast<int *>(base + k::kOffRows);
        k::k_noalloc_front<<<k::cdiv(k, 128), 128, 0, s>>>(k, i64, i32, rows);
        HSIM_LAUNCHED();
        k::FrontDev fd{i64 + 0, i32 + 0, i32 + 1, i32 + 2, i64 + 2, rows, i64 + 4, i32 + 3};
        int flag_host[4] = {0, 0, 0, 0};
        int sw = 0;
        int rc = k::ritz_on(s, k, Sbar_dev, k, Mbar_dev, k, evals_dev, X_dev, k, work, fd, i32 + 4, &sw, i32 + 8,
                            flag_host);
        HSIM_CUDA(cudaStreamSynchronize(s));
        if (sweeps_out) *sweeps_out = sw;
        if (rc == 1) fail(HSIM_E_NOT_SPD, "M_bar is not positive definite");
        if (rc == 2)
            fail(HSIM_E_NO_CONVERGENCE, "hsim_ritz_noalloc: Jacobi sweeps still rotating after " +
                                            std::to_string(sw) + " sweeps");
        return HSIM_OK;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return HSIM_E_INTERNAL;
    }
}
