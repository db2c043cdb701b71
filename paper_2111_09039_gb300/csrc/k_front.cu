// Multifrontal LDL^T factorisation of the shifted level matrix and its
// multi-right-hand-side solves (Alg. 1: one factorisation of S - mu M per
// level, then (S - mu M) Psi = M Phi for all q columns; Sec. 3.2 "Direct
// solver": symmetric indefinite LDL^T).
//
// Every front is a dense column-major nf x nf block of one arena; its first
// ns columns are the pivots.  Fronts of equal height in the elimination tree
// are independent and are processed by the same launches.  A front is
// factored in panels of kPanel = 32 columns (right-looking):
//   diag:    LDL^T of the 32 x 32 diagonal block in shared memory (one CTA
//            per front), written back in place;
//   panel:   L21 = A21 L11^-T D^-1, one tile of 128 rows per CTA;
//   update:  A22 -= L21 D L21^T on lower-triangular 64 x 64 tiles;
// and the children's update blocks are added into the parent front
// (extend-add) before the parent is factored.  Pivoting is not used: the
// shifted Laplacian is factored as is after the fill-reducing ordering; a
// pivot below the tolerance is reported and replaced by +-tol.
//
// The solves work on row-major X (n x k, internal order) so that each row
// of a right-hand-side block is a contiguous, coalesced segment.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>

#include "common.h"
#include "host.h"
#include "kernels.h"

namespace hsim {
namespace k {

namespace {

constexpr int P = kPanel;  // 32

__device__ __forceinline__ void tri_index(int64_t x, int &ti, int &tj) {
    // x -> (ti, tj) with ti >= tj, x = ti (ti + 1) / 2 + tj
    int t = (int)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
    while ((int64_t)t * (t + 1) / 2 > x) --t;
    while ((int64_t)(t + 1) * (t + 2) / 2 <= x) ++t;
    ti = t;
    tj = (int)(x - (int64_t)t * (t + 1) / 2);
}

template <typename T>
__global__ void k_front_assemble(int64_t nnz, const int *__restrict__ row_of, const int *__restrict__ col,
                                 const int64_t *__restrict__ dst, const double *__restrict__ S,
                                 const double *__restrict__ M, const double *__restrict__ Md, double mu,
                                 T *__restrict__ arena) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    int64_t d = dst[e];
    if (d < 0) return;
    double v = S[e];
    if (M) {
        v -= mu * M[e];
    } else {
        int r = row_of[e];
        if (r == col[e]) v -= mu * Md[r];
    }
    arena[d] = (T)v;
}

// extend-add of the update blocks of `children` into their parents
template <typename T>
__global__ void k_extend_add(FrontDev fd, const int *__restrict__ parent, const int *__restrict__ children,
                             T *__restrict__ arena) {
    const int c = children[blockIdx.x];
    const int nsc = fd.ns[c], nfc = fd.nf[c];
    const int u = nfc - nsc;
    const int nt = (u + 31) / 32;
    int ti, tj;
    tri_index(blockIdx.y, ti, tj);
    if (ti >= nt) return;
    const int p = parent[c];
    const int nfp = fd.nf[p];
    const int *rel = fd.relmap + fd.relmap_off[c];
    const T *Fc = arena + fd.foff[c];
    T *Fp = arena + fd.foff[p];
    const int jl = threadIdx.x & 31;
    const int j = tj * 32 + jl;
    if (j >= u) return;
    const int pj = rel[j];
    for (int il = threadIdx.x >> 5; il < 32; il += blockDim.x >> 5) {
        int i = ti * 32 + il;
        if (i >= u || i < j) continue;
        T v = Fc[(int64_t)(nsc + j) * nfc + (nsc + i)];
        if (v != T(0)) atomicAdd(&Fp[(int64_t)pj * nfp + rel[i]], v);
    }
}

// Factor the kb x kb diagonal block held in smem column-major D[c][r]
// (LDL^T, unit L below the diagonal, D on the diagonal).
template <typename T>
__device__ void ldlt_block(T (*Dg)[P + 1], int kb, double tol, int *flags) {
    __shared__ T lj[P];
    for (int j = 0; j < kb; ++j) {
        __syncthreads();
        T d = Dg[j][j];
        if (!(fabs((double)d) >= tol)) {  // also catches NaN
            if (threadIdx.x == 0) atomicAdd(&flags[0], 1);
            d = (d < T(0)) ? (T)-tol : (T)tol;
        }
        for (int i = j + 1 + threadIdx.x; i < kb; i += blockDim.x) lj[i] = Dg[j][i] / d;
        __syncthreads();
        for (int idx = threadIdx.x; idx < (kb - j - 1) * (kb - j - 1); idx += blockDim.x) {
            int r = j + 1 + idx % (kb - j - 1);
            int c = j + 1 + idx / (kb - j - 1);
            if (r >= c) Dg[c][r] -= lj[r] * d * lj[c];
        }
        __syncthreads();
        if (threadIdx.x == 0) Dg[j][j] = d;
        for (int i = j + 1 + threadIdx.x; i < kb; i += blockDim.x) Dg[j][i] = lj[i];
    }
    __syncthreads();
}

constexpr int kPanelRows = 128;

// LDL^T of the kb x kb diagonal block of panel k0, one CTA per front,
// written back in place (unit L below the diagonal, D on it).
template <typename T>
__global__ void __launch_bounds__(128) k_front_diag_block(FrontDev fd, const int *__restrict__ nodes, int k0,
                                                          T *__restrict__ arena, double tol, int *flags) {
    __shared__ T Dg[P][P + 1];
    const int t = nodes[blockIdx.x];
    const int nf = fd.nf[t], ns = fd.ns[t];
    const int kb = min(P, ns - k0);
    if (kb <= 0) return;
    T *F = arena + fd.foff[t];
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        int r = idx % kb, c = idx / kb;
        Dg[c][r] = (r >= c) ? F[(int64_t)(k0 + c) * nf + (k0 + r)] : 0.0;
    }
    ldlt_block(Dg, kb, tol, flags);
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        int r = idx % kb, c = idx / kb;
        if (r >= c) F[(int64_t)(k0 + c) * nf + (k0 + r)] = Dg[c][r];
    }
}

// Rows below the diagonal block: x L11^T = a, l = x / d, with L11 and D
// read from the block factored by k_front_diag_block in the previous launch.
template <typename T>
__global__ void __launch_bounds__(128) k_front_panel(FrontDev fd, const int *__restrict__ nodes, int k0,
                                                     T *__restrict__ arena) {
    __shared__ T Dg[P][P + 1];
    const int t = nodes[blockIdx.x];
    const int nf = fd.nf[t], ns = fd.ns[t];
    const int kb = min(P, ns - k0);
    if (kb <= 0) return;
    const int r0 = k0 + kb + blockIdx.y * kPanelRows;
    if (r0 >= nf) return;
    T *F = arena + fd.foff[t];
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        int r = idx % kb, c = idx / kb;
        Dg[c][r] = (r >= c) ? F[(int64_t)(k0 + c) * nf + (k0 + r)] : 0.0;
    }
    __syncthreads();
    const int r = r0 + threadIdx.x;
    if (r < nf) {
        T x[P];
#pragma unroll
        for (int c = 0; c < P; ++c)
            if (c < kb) x[c] = F[(int64_t)(k0 + c) * nf + r];
#pragma unroll
        for (int c = 0; c < P; ++c) {
            if (c < kb) {
                T v = x[c];
#pragma unroll
                for (int cc = 0; cc < P; ++cc)
                    if (cc < c) v -= x[cc] * Dg[cc][c];
                x[c] = v;
            }
        }
#pragma unroll
        for (int c = 0; c < P; ++c)
            if (c < kb) F[(int64_t)(k0 + c) * nf + r] = x[c] / Dg[c][c];
    }
}

// A22 -= L21 D L21^T on 64 x 64 lower-triangular tiles of the trailing block;
// with ntj > 0 only the columns below c_end (tile y = ti * ntj + tj)
template <typename T>
__global__ void __launch_bounds__(256) k_front_update(FrontDev fd, const int *__restrict__ nodes, int k0,
                                                      T *__restrict__ arena, int c_end, int ntj) {
    __shared__ T Lr[P][64];
    __shared__ T Lc[P][64];
    const int t = nodes[blockIdx.x];
    const int nf = fd.nf[t], ns = fd.ns[t];
    const int kb = min(P, ns - k0);
    if (kb <= 0) return;
    const int base = k0 + kb;
    const int m = nf - base;
    if (m <= 0) return;
    const int nt = (m + 63) / 64;
    int ti, tj;
    if (ntj > 0) {
        ti = (int)(blockIdx.y / ntj);
        tj = (int)(blockIdx.y % ntj);
        if (ti < tj) return;
    } else {
        tri_index(blockIdx.y, ti, tj);
    }
    if (ti >= nt) return;
    T *F = arena + fd.foff[t];
    const int r0 = base + ti * 64, c0 = base + tj * 64;
    if (c0 >= c_end) return;
    for (int idx = threadIdx.x; idx < P * 64; idx += blockDim.x) {
        int i = idx & 63, kk = idx >> 6;
        T vr = 0.0, vc = 0.0;
        if (kk < kb) {
            T d = F[(int64_t)(k0 + kk) * nf + (k0 + kk)];
            if (r0 + i < nf) vr = F[(int64_t)(k0 + kk) * nf + (r0 + i)];
            if (c0 + i < nf) vc = F[(int64_t)(k0 + kk) * nf + (c0 + i)] * d;
        }
        Lr[kk][i] = vr;
        Lc[kk][i] = vc;
    }
    __syncthreads();
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4] = {};
    for (int kk = 0; kk < kb; ++kk) {
        T a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] = Lr[kk][ty + 16 * u];
            b[u] = Lc[kk][tx + 16 * u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int r = r0 + ty + 16 * u;
        if (r >= nf) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int c = c0 + tx + 16 * v;
            if (c < nf && r >= c && c < c_end) F[(int64_t)c * nf + r] -= acc[u][v];
        }
    }
}

template <typename T>
__global__ void k_front_diag(FrontDev fd, const int *__restrict__ nodes, int n_nodes,
                             const T *__restrict__ arena, T *__restrict__ dpos, int *neg) {
    int t_idx = blockIdx.x;
    if (t_idx >= n_nodes) return;
    int t = nodes[t_idx];
    const int nf = fd.nf[t], ns = fd.ns[t], ps = fd.pstart[t];
    const T *F = arena + fd.foff[t];
    int cnt = 0;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        T d = F[(int64_t)i * nf + i];
        dpos[ps + i] = d;
        cnt += (d < T(0));
    }
    if (cnt) atomicAdd(neg, cnt);
}

template <typename T>
__global__ void k_front_maxdiag(FrontDev fd, const T *__restrict__ arena, unsigned long long *out) {
    const int t = blockIdx.x;
    const int nf = fd.nf[t], ns = fd.ns[t];
    const T *F = arena + fd.foff[t];
    unsigned long long best = 0;
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        unsigned long long b = (unsigned long long)__double_as_longlong(fabs((double)F[(int64_t)i * nf + i]));
        best = b > best ? b : best;
    }
    if (best) atomicMax(out, best);
}

// ---- solves ---------------------------------------------------------------
constexpr int kTriCols = 128;

// X[panel rows, cols] = L11^-1 X[...]  (unit lower, forward)
template <typename T>
__global__ void __launch_bounds__(kTriCols) k_solve_fwd_tri(FrontDev fd, const int *__restrict__ nodes, int k0,
                                                            const T *__restrict__ arena, int k,
                                                            T *__restrict__ X, int ldx) {
    __shared__ T L[P][P + 1];
    const int t = nodes[blockIdx.x];
    const int nf = fd.nf[t], ns = fd.ns[t], ps = fd.pstart[t];
    const int kb = min(P, ns - k0);
    if (kb <= 0) return;
    const T *F = arena + fd.foff[t];
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        int r = idx % kb, c = idx / kb;
        L[r][c] = (r > c) ? F[(int64_t)(k0 + c) * nf + (k0 + r)] : 0.0;
    }
    __syncthreads();
    const int j = blockIdx.y * kTriCols + threadIdx.x;
    if (j >= k) return;
    T x[P];
    T *Xb = X + (size_t)(ps + k0) * ldx + j;
#pragma unroll
    for (int r = 0; r < P; ++r)
        if (r < kb) x[r] = Xb[(size_t)r * ldx];
#pragma unroll
    for (int r = 1; r < P; ++r) {
        if (r < kb) {
            T v = x[r];
#pragma unroll
            for (int c = 0; c < P; ++c)
                if (c < r) v -= L[r][c] * x[c];
            x[r] = v;
        }
    }
#pragma unroll
    for (int r = 0; r < P; ++r)
        if (r < kb) Xb[(size_t)r * ldx] = x[r];
}

// x[0..3] -= a[0..3] with atomics (one vector atomic for four aligned floats)
__device__ __forceinline__ void atomic_sub4(float *x, const float (&a)[4], int avail) {
    if (avail >= 4 && (reinterpret_cast<uintptr_t>(x) & 15u) == 0) {
        atomicAdd(reinterpret_cast<float4 *>(x), make_float4(-a[0], -a[1], -a[2], -a[3]));
    } else {
        for (int v = 0; v < 4 && v < avail; ++v) atomicAdd(x + v, -a[v]);
    }
}
__device__ __forceinline__ void atomic_sub4(double *x, const double (&a)[4], int avail) {
    for (int v = 0; v < 4 && v < avail; ++v) atomicAdd(x + v, -a[v]);
}

// X[row(r), cols] -= sum_c L[r, k0+c] X[panel row c, cols] for front rows
// r >= k0 + kb; pivot rows of the front are updated in place, rows of
// ancestor fronts with atomics (sibling fronts share them).
template <typename T>
__global__ void __launch_bounds__(256) k_solve_fwd_upd(FrontDev fd, const int *__restrict__ nodes, int k0,
                                                       const T *__restrict__ arena, int k,
                                                       T *__restrict__ X, int ldx) {
    __shared__ T Ls[P][64];
    __shared__ T Xs[P][64];
    const int t = nodes[blockIdx.x];
    const int nf = fd.nf[t], ns = fd.ns[t], ps = fd.pstart[t];
    const int kb = min(P, ns - k0);
    if (kb <= 0) return;
    const int base = k0 + kb;
    const int r0 = base + blockIdx.y * 64;
    if (r0 >= nf) return;
    const int c0 = blockIdx.z * 64;
    if (c0 >= k) return;
    const T *F = arena + fd.foff[t];
    const int *rows = fd.rows + fd.rows_off[t];
    for (int idx = threadIdx.x; idx < P * 64; idx += blockDim.x) {
        int i = idx & 63, kk = idx >> 6;
        T lv = 0.0, xv = 0.0;
        if (kk < kb) {
            if (r0 + i < nf) lv = F[(int64_t)(k0 + kk) * nf + (r0 + i)];
            if (c0 + i < k) xv = X[(size_t)(ps + k0 + kk) * ldx + c0 + i];
        }
        Ls[kk][i] = lv;
        Xs[kk][i] = xv;
    }
    __syncthreads();
    // thread: rows ty + 16 u, four contiguous columns 4 tx .. 4 tx + 3
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[4][4] = {};
    for (int kk = 0; kk < kb; ++kk) {
        T a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            a[u] = Ls[kk][ty + 16 * u];
            b[u] = Xs[kk][4 * tx + u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    const int cb = c0 + 4 * tx;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int r = r0 + ty + 16 * u;
        if (r >= nf) continue;
        int grow = rows[r];
        T *xr = X + (size_t)grow * ldx + cb;
        if (r < ns) {
#pragma unroll
            for (int v = 0; v < 4; ++v)
                if (cb + v < k) xr[v] -= acc[u][v];
        } else {
            atomic_sub4(xr, acc[u], k - cb);
        }
    }
}

template <typename T>
__global__ void k_solve_diag(int n, int k, const T *__restrict__ dpos, T *__restrict__ X, int ldx) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * k) return;
    int i = (int)(idx / k), j = (int)(idx % k);
    X[(size_t)i * ldx + j] /= dpos[i];
}

// X[panel rows c, cols] -= sum_{r >= k0+kb} L[r, k0+c] X[row(r), cols].  A CTA
// covers kBwdChunks 32-row chunks of r; when one CTA covers all rows of the
// front (grid.y == 1) it updates the panel rows with plain stores, otherwise
// the partial sums are accumulated with atomics.
constexpr int kBwdChunks = 1;
template <typename T>
__global__ void __launch_bounds__(256) k_solve_bwd_upd(FrontDev fd, const int *__restrict__ nodes, int k0,
                                                       const T *__restrict__ arena, int k,
                                                       T *__restrict__ X, int ldx) {
    __shared__ T Ls[P][P + 1];  // [r][c]
    __shared__ T Xs[P][64];     // [r][col]
    const int t = nodes[blockIdx.x];
    const int nf = fd.nf[t], ns = fd.ns[t], ps = fd.pstart[t];
    const int kb = min(P, ns - k0);
    if (kb <= 0) return;
    const int base = k0 + kb;
    const int rbeg = base + blockIdx.y * P * kBwdChunks;
    if (rbeg >= nf) return;
    const int rend = min(nf, rbeg + P * kBwdChunks);
    const int c0 = blockIdx.z * 64;
    if (c0 >= k) return;
    const T *F = arena + fd.foff[t];
    const int *rows = fd.rows + fd.rows_off[t];
    // 32 x 64 outputs, 8 per thread: thread -> column j = tid & 63, rows c = (tid >> 6) + 4u
    const int j = threadIdx.x & 63, cb = threadIdx.x >> 6;
    T acc[8] = {};
    for (int r0 = rbeg; r0 < rend; r0 += P) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < P * P; idx += blockDim.x) {
            int r = idx % P, c = idx / P;
            Ls[r][c] = (r0 + r < rend && c < kb) ? F[(int64_t)(k0 + c) * nf + (r0 + r)] : T(0);
        }
        for (int idx = threadIdx.x; idx < P * 64; idx += blockDim.x) {
            int jj = idx & 63, r = idx >> 6;
            Xs[r][jj] = (r0 + r < rend && c0 + jj < k) ? X[(size_t)rows[r0 + r] * ldx + c0 + jj] : T(0);
        }
        __syncthreads();
        for (int r = 0; r < P; ++r) {
            T xv = Xs[r][j];
#pragma unroll
            for (int u = 0; u < 8; ++u) acc[u] += Ls[r][cb + 4 * u] * xv;
        }
    }
    if (c0 + j < k) {
        const bool whole = gridDim.y == 1;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            int c = cb + 4 * u;
            if (c < kb) {
                T *x = &X[(size_t)(ps + k0 + c) * ldx + c0 + j];
                if (whole) *x -= acc[u];
                else atomicAdd(x, -acc[u]);
            }
        }
    }
}

// X[panel rows, cols] = L11^-T X[...]  (unit upper, backward)
template <typename T>
__global__ void __launch_bounds__(kTriCols) k_solve_bwd_tri(FrontDev fd, const int *__restrict__ nodes, int k0,
                                                            const T *__restrict__ arena, int k,
                                                            T *__restrict__ X, int ldx) {
    __shared__ T L[P][P + 1];
    const int t = nodes[blockIdx.x];
    const int nf = fd.nf[t], ns = fd.ns[t], ps = fd.pstart[t];
    const int kb = min(P, ns - k0);
    if (kb <= 0) return;
    const T *F = arena + fd.foff[t];
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
        int r = idx % kb, c = idx / kb;
        L[r][c] = (r > c) ? F[(int64_t)(k0 + c) * nf + (k0 + r)] : 0.0;
    }
    __syncthreads();
    const int j = blockIdx.y * kTriCols + threadIdx.x;
    if (j >= k) return;
    T x[P];
    T *Xb = X + (size_t)(ps + k0) * ldx + j;
#pragma unroll
    for (int r = 0; r < P; ++r)
        if (r < kb) x[r] = Xb[(size_t)r * ldx];
#pragma unroll
    for (int r = P - 2; r >= 0; --r) {
        if (r < kb - 1) {
            T v = x[r];
#pragma unroll
            for (int c = 0; c < P; ++c)
                if (c > r && c < kb) v -= L[c][r] * x[c];
            x[r] = v;
        }
    }
#pragma unroll
    for (int r = 0; r < P; ++r)
        if (r < kb) Xb[(size_t)r * ldx] = x[r];
}

// ---- single-panel fronts (ns <= P, nf <= kSmallNf): fused solve kernels -------
// One CTA per (front, column tile): the front's L panel and pivot rows are
// staged in shared memory once; the forward kernel solves the unit lower
// triangle and sends L21 x1 to the ancestors' rows (vector atomics), the
// backward kernel gathers the ancestors' rows, subtracts L21^T x2 and solves
// the unit upper triangle.  Thread layout for the products: 4 contiguous
// columns per thread, 8 row groups.
template <typename T>
__host__ __device__ constexpr int small_cols() { return 512 / (int)sizeof(T); }  // 128 float, 64 double

// copy n values of one row between global and shared memory: 16-byte vectors
// when `vec` (both addresses 16-byte aligned, n a multiple of the vector)
template <typename T>
__device__ __forceinline__ void row_load(T *dst, const T *src, int n, int lane, int lanes, bool vec) {
    constexpr int V = 16 / (int)sizeof(T);
    if (vec && n % V == 0) {
        for (int i = lane; i < n / V; i += lanes) reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(src)[i];
    } else {
        for (int i = lane; i < n; i += lanes) dst[i] = src[i];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_solve_fwd_small(FrontDev fd, const int *__restrict__ nodes,
                                                         const T *__restrict__ arena, int k, T *__restrict__ X,
                                                         int ldx, bool vec, int nf_max) {
    constexpr int SC = small_cols<T>();
    constexpr int CG = SC / 4;   // column groups of 4
    constexpr int RG = 256 / CG; // row groups
    extern __shared__ __align__(16) unsigned char small_smem[];
    T *Ls = reinterpret_cast<T *>(small_smem);  // ns x nf (column-major panel)
    T *Xp = Ls + P * nf_max;                    // [P][SC]
    const int t = nodes[blockIdx.x];
    const int nf = fd.nf[t], ns = fd.ns[t], ps = fd.pstart[t];
    const int c0 = blockIdx.y * SC;
    if (c0 >= k) return;
    const int tid = threadIdx.x;
    const T *F = arena + fd.foff[t];
    for (int i = tid; i < ns * nf; i += 256) Ls[i] = F[i];
    const int cols = min(SC, k - c0);
    // pivot rows: one warp per row
    for (int r = tid / 32; r < ns; r += 8) {
        row_load(Xp + r * SC, X + (size_t)(ps + r) * ldx + c0, cols, tid % 32, 32, vec);
        for (int c = cols + tid % 32; c < SC; c += 32) Xp[r * SC + c] = T(0);
    }
    __syncthreads();
    if (tid < SC) {
        for (int r = 1; r < ns; ++r) {
            T acc = Xp[r * SC + tid];
            for (int q = 0; q < r; ++q) acc -= Ls[q * nf + r] * Xp[q * SC + tid];
            Xp[r * SC + tid] = acc;
        }
    }
    __syncthreads();
    for (int r = tid / 32; r < ns; r += 8) row_load(X + (size_t)(ps + r) * ldx + c0, Xp + r * SC, cols, tid % 32, 32, vec);
    // ancestors' rows: x_r -= L_r. x_p
    const int cg = (tid % CG) * 4, rg = tid / CG;
    const int *rows = fd.rows + fd.rows_off[t];
    for (int r = ns + rg; r < nf; r += RG) {
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int q = 0; q < ns; ++q) {
            const T l = Ls[q * nf + r];
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[v] += l * Xp[q * SC + cg + v];
        }
        atomic_sub4(X + (size_t)rows[r] * ldx + c0 + cg, acc, k - c0 - cg);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_solve_bwd_small(FrontDev fd, const int *__restrict__ nodes,
                                                         const T *__restrict__ arena, int k, T *__restrict__ X,
                                                         int ldx, bool vec, int nf_max) {
    constexpr int SC = small_cols<T>();
    constexpr int CG = SC / 4;
    constexpr int RG = 256 / CG;
    extern __shared__ __align__(16) unsigned char small_smem[];
    T *Ls = reinterpret_cast<T *>(small_smem);
    T *Xp = Ls + P * nf_max;    // [P][SC]
    T *Xu = Xp + P * SC;        // [P][SC] chunk of ancestor rows
    const int t = nodes[blockIdx.x];
    const int nf = fd.nf[t], ns = fd.ns[t], ps = fd.pstart[t];
    const int c0 = blockIdx.y * SC;
    if (c0 >= k) return;
    const int tid = threadIdx.x;
    const T *F = arena + fd.foff[t];
    const int *rows = fd.rows + fd.rows_off[t];
    for (int i = tid; i < ns * nf; i += 256) Ls[i] = F[i];
    const int cols = min(SC, k - c0);
    for (int r = tid / 32; r < ns; r += 8) {
        row_load(Xp + r * SC, X + (size_t)(ps + r) * ldx + c0, cols, tid % 32, 32, vec);
        for (int c = cols + tid % 32; c < SC; c += 32) Xp[r * SC + c] = T(0);
    }
    // x_p -= L21^T x_u over 32-row chunks of the ancestors' rows; thread: pivots
    // q = rg + RG j, columns cg .. cg + 3
    const int cg = (tid % CG) * 4, rg = tid / CG;
    constexpr int QJ = (P + RG - 1) / RG;
    T acc[QJ][4];
#pragma unroll
    for (int j = 0; j < QJ; ++j)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[j][v] = T(0);
    for (int r0 = ns; r0 < nf; r0 += P) {
        const int cnt = min(P, nf - r0);
        __syncthreads();
        for (int rr = tid / 32; rr < cnt; rr += 8) {
            row_load(Xu + rr * SC, X + (size_t)rows[r0 + rr] * ldx + c0, cols, tid % 32, 32, vec);
            for (int c = cols + tid % 32; c < SC; c += 32) Xu[rr * SC + c] = T(0);
        }
        __syncthreads();
        for (int rr = 0; rr < cnt; ++rr) {
            T xu[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) xu[v] = Xu[rr * SC + cg + v];
#pragma unroll
            for (int j = 0; j < QJ; ++j) {
                const int q = rg + RG * j;
                if (q < ns) {
                    const T l = Ls[q * nf + r0 + rr];
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[j][v] += l * xu[v];
                }
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < QJ; ++j) {
        const int q = rg + RG * j;
        if (q < ns)
#pragma unroll
            for (int v = 0; v < 4; ++v) Xp[q * SC + cg + v] -= acc[j][v];
    }
    __syncthreads();
    if (tid < SC) {
        for (int r = ns - 2; r >= 0; --r) {
            T a = Xp[r * SC + tid];
            for (int q = r + 1; q < ns; ++q) a -= Ls[r * nf + q] * Xp[q * SC + tid];
            Xp[r * SC + tid] = a;
        }
    }
    __syncthreads();
    for (int r = tid / 32; r < ns; r += 8) row_load(X + (size_t)(ps + r) * ldx + c0, Xp + r * SC, cols, tid % 32, 32, vec);
}

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

template <typename T>
void front_assemble(cudaStream_t s, int64_t nnz, const int *row_of, const int *col, const int64_t *dst,
                    const double *S_val, const double *M_val, const double *M_diag, double mu, T *arena) {
    if (nnz <= 0) return;
    k_front_assemble<T><<<cdiv(nnz, 256), 256, 0, s>>>(nnz, row_of, col, dst, S_val, M_val, M_diag, mu, arena);
    HSIM_LAUNCHED();
}

template <typename T>
void front_extend_add(cudaStream_t s, const FrontDev &fd, const int *parent, const int *children, int n_children,
                      int max_upd, T *arena) {
    if (n_children <= 0 || max_upd <= 0) return;
    int64_t Tt = (max_upd + 31) / 32;
    dim3 g((unsigned)n_children, (unsigned)(Tt * (Tt + 1) / 2));
    k_extend_add<T><<<g, 256, 0, s>>>(fd, parent, children, arena);
    HSIM_LAUNCHED();
}

template <typename T>
void front_panel(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0, int max_rows, T *arena,
                 double pivot_tol, int *flags) {
    if (n_nodes <= 0) return;
    k_front_diag_block<T><<<(unsigned)n_nodes, 128, 0, s>>>(fd, nodes, k0, arena, pivot_tol, flags);
    HSIM_LAUNCHED();
    if (max_rows <= 0) return;
    dim3 g((unsigned)n_nodes, cdiv(max_rows, kPanelRows));
    k_front_panel<T><<<g, 128, 0, s>>>(fd, nodes, k0, arena);
    HSIM_LAUNCHED();
}

template <typename T>
void front_update(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0, int max_trail, T *arena,
                  int c_end) {
    if (n_nodes <= 0 || max_trail <= 0) return;
    int64_t Tt = (max_trail + 63) / 64;
    // column tiles below c_end (the trailing part starts after k0's first pivot)
    const int64_t ntj = c_end == INT_MAX ? 0 : std::min<int64_t>(Tt, (c_end - k0 + 62) / 64 + 1);
    if (c_end != INT_MAX && ntj <= 0) return;
    dim3 g((unsigned)n_nodes, (unsigned)(ntj > 0 ? Tt * ntj : Tt * (Tt + 1) / 2));
    k_front_update<T><<<g, 256, 0, s>>>(fd, nodes, k0, arena, c_end, (int)ntj);
    HSIM_LAUNCHED();
}

template <typename T>
void front_maxdiag(cudaStream_t s, const FrontDev &fd, int n_nodes, const T *arena, unsigned long long *out) {
    if (n_nodes <= 0) return;
    k_front_maxdiag<T><<<n_nodes, 128, 0, s>>>(fd, arena, out);
    HSIM_LAUNCHED();
}

template <typename T>
void front_diag(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, const T *arena, T *dpos,
                int *neg_count) {
    if (n_nodes <= 0) return;
    k_front_diag<T><<<n_nodes, 128, 0, s>>>(fd, nodes, n_nodes, arena, dpos, neg_count);
    HSIM_LAUNCHED();
}

template <typename T>
void solve_fwd_tri(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0, const T *arena, int k,
                   T *X, int ldx) {
    if (n_nodes <= 0 || k <= 0) return;
    dim3 g((unsigned)n_nodes, cdiv(k, kTriCols));
    k_solve_fwd_tri<T><<<g, kTriCols, 0, s>>>(fd, nodes, k0, arena, k, X, ldx);
    HSIM_LAUNCHED();
}

template <typename T>
void solve_fwd_upd(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0, int max_rows,
                   const T *arena, int k, T *X, int ldx) {
    if (n_nodes <= 0 || k <= 0 || max_rows <= 0) return;
    dim3 g((unsigned)n_nodes, cdiv(max_rows, 64), cdiv(k, 64));
    k_solve_fwd_upd<T><<<g, 256, 0, s>>>(fd, nodes, k0, arena, k, X, ldx);
    HSIM_LAUNCHED();
}

template <typename T>
void solve_diag(cudaStream_t s, int n, int k, const T *dpos, T *X, int ldx) {
    if (n <= 0 || k <= 0) return;
    k_solve_diag<T><<<cdiv((int64_t)n * k, 256), 256, 0, s>>>(n, k, dpos, X, ldx);
    HSIM_LAUNCHED();
}

template <typename T>
void solve_bwd_upd(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0, int max_rows,
                   const T *arena, int k, T *X, int ldx) {
    if (n_nodes <= 0 || k <= 0 || max_rows <= 0) return;
    dim3 g((unsigned)n_nodes, cdiv(max_rows, P * kBwdChunks), cdiv(k, 64));
    k_solve_bwd_upd<T><<<g, 256, 0, s>>>(fd, nodes, k0, arena, k, X, ldx);
    HSIM_LAUNCHED();
}

template <typename T>
void solve_bwd_tri(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int k0, const T *arena, int k,
                   T *X, int ldx) {
    if (n_nodes <= 0 || k <= 0) return;
    dim3 g((unsigned)n_nodes, cdiv(k, kTriCols));
    k_solve_bwd_tri<T><<<g, kTriCols, 0, s>>>(fd, nodes, k0, arena, k, X, ldx);
    HSIM_LAUNCHED();
}

template <typename T>
void solve_fwd_small(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int nf_max, const T *arena,
                     int k, T *X, int ldx) {
    if (n_nodes <= 0 || k <= 0) return;
    nf_max = (nf_max + 3) & ~3;  // keeps the row blocks after the panel 16-byte aligned
    const size_t sm = ((size_t)P * nf_max + (size_t)P * small_cols<T>()) * sizeof(T);
    HSIM_SMEM_LIMIT_ONCE(k_solve_fwd_small<T>, ((size_t)P * kSmallNf + (size_t)P * small_cols<T>()) * sizeof(T));
    const bool vec = (reinterpret_cast<uintptr_t>(X) % 16 == 0) && ((size_t)ldx * sizeof(T)) % 16 == 0;
    k_solve_fwd_small<T><<<dim3((unsigned)n_nodes, cdiv(k, small_cols<T>())), 256, sm, s>>>(fd, nodes, arena, k, X,
                                                                                             ldx, vec, nf_max);
    HSIM_LAUNCHED();
}

template <typename T>
void solve_bwd_small(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int nf_max, const T *arena,
                     int k, T *X, int ldx) {
    if (n_nodes <= 0 || k <= 0) return;
    nf_max = (nf_max + 3) & ~3;
    const size_t sm = ((size_t)P * nf_max + 2 * (size_t)P * small_cols<T>()) * sizeof(T);
    HSIM_SMEM_LIMIT_ONCE(k_solve_bwd_small<T>,
                         ((size_t)P * kSmallNf + 2 * (size_t)P * small_cols<T>()) * sizeof(T));
    const bool vec = (reinterpret_cast<uintptr_t>(X) % 16 == 0) && ((size_t)ldx * sizeof(T)) % 16 == 0;
    k_solve_bwd_small<T><<<dim3((unsigned)n_nodes, cdiv(k, small_cols<T>())), 256, sm, s>>>(fd, nodes, arena, k, X,
                                                                                             ldx, vec, nf_max);
    HSIM_LAUNCHED();
}

#define HSIM_FRONT_INSTANTIATE(T)                                                                                  \
    template void front_assemble<T>(cudaStream_t, int64_t, const int *, const int *, const int64_t *,            \
                                    const double *, const double *, const double *, double, T *);               \
    template void front_extend_add<T>(cudaStream_t, const FrontDev &, const int *, const int *, int, int, T *);  \
    template void front_panel<T>(cudaStream_t, const FrontDev &, const int *, int, int, int, T *, double, int *);  \
    template void front_update<T>(cudaStream_t, const FrontDev &, const int *, int, int, int, T *, int);         \
    template void front_maxdiag<T>(cudaStream_t, const FrontDev &, int, const T *, unsigned long long *);        \
    template void front_diag<T>(cudaStream_t, const FrontDev &, const int *, int, const T *, T *, int *);        \
    template void solve_fwd_tri<T>(cudaStream_t, const FrontDev &, const int *, int, int, const T *, int, T *, int); \
    template void solve_fwd_upd<T>(cudaStream_t, const FrontDev &, const int *, int, int, int, const T *, int, T *, \
                                   int);                                                                         \
    template void solve_diag<T>(cudaStream_t, int, int, const T *, T *, int);                                    \
    template void solve_bwd_upd<T>(cudaStream_t, const FrontDev &, const int *, int, int, int, const T *, int, T *, \
                                   int);                                                                         \
    template void solve_bwd_tri<T>(cudaStream_t, const FrontDev &, const int *, int, int, const T *, int, T *, int); \
    template void solve_fwd_small<T>(cudaStream_t, const FrontDev &, const int *, int, int, const T *, int, T *, int); \
    template void solve_bwd_small<T>(cudaStream_t, const FrontDev &, const int *, int, int, const T *, int, T *, int);

HSIM_FRONT_INSTANTIATE(float)
HSIM_FRONT_INSTANTIATE(double)

}  // namespace k
}  // namespace hsim
