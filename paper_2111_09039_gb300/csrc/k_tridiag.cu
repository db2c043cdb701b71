// Dense symmetric eigensolver (FP64) for the Rayleigh-Ritz problems of Alg. 1
// and the coarsest-level problem of Alg. 3: the lowest m eigenpairs of a
// symmetric n x n matrix A.
//
//   1. Householder tridiagonalisation Q^T A Q = T in one cooperative launch:
//      per column k every CTA rebuilds the reflector v_k = (1, x_2..)/(x_1 -
//      beta) from the column below the diagonal (so no barrier is needed to
//      share it), computes p = tau A22 v over its rows of the trailing block,
//      forms w = p - (tau/2)(p.v) v and applies A22 -= v w^T + w v^T to its
//      rows.  Where the matrix fits in the CTAs' shared memory (n up to about
//      1650 on 152 SMs) each CTA keeps its rows there and one grid barrier per
//      column suffices (k_tridiag_rows); otherwise the rows stay in global
//      memory with two barriers per column (k_tridiag).  The reflectors are
//      kept row-wise in Vh (contiguous for the back transformation).
//   2. Eigenvalues of T by multisection on Sturm counts, one warp per index
//      (ascending by construction): FP32 rounds, an FP64 check of the
//      bracket, FP64 rounds.
//   3. Eigenvectors of T by inverse iteration on T - lambda I (Gaussian
//      elimination with partial pivoting, reciprocal pivots kept), three
//      iterations from a hashed random start; eigenvalues closer than
//      1e-5 ||T|| form a cluster whose vectors are made orthogonal to the
//      previous ones of the cluster in every iteration (one warp per cluster).
//   4. Back transformation X = Q Z, reflectors applied in reverse order: one
//      warp per eigenvector held in registers (n <= 2048), else a few
//      eigenvectors per CTA held in shared memory.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "common.h"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace hsim {
namespace k {

namespace {

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

constexpr int kTriThreads = 256;
constexpr double kClusterTol = 1e-5;  // relative to ||T||
constexpr size_t kTriSmemMax = 200 * 1024;  // dynamic shared memory limit of k_tridiag and k_tri_back

// sum over the block (256 threads); `red` holds 8 doubles; result in all threads
__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5;
    __syncthreads();  // red may still be read from the previous call
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < kTriThreads / 32; ++i) s += red[i];
    return s;
}

__global__ void __launch_bounds__(kTriThreads) k_tridiag(int n, double *__restrict__ A, double *__restrict__ d,
                                                       double *__restrict__ e, double *__restrict__ tau,
                                                       double *__restrict__ Vh, double *__restrict__ p) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ double sm[];
    double *v = sm;       // n
    double *w = sm + n;   // n
    __shared__ double red[kTriThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31;
    const int gwarp = (blockIdx.x * kTriThreads + tid) >> 5, nwarps = gridDim.x * (kTriThreads / 32);
    for (int k = 0; k + 1 < n; ++k) {
        const int L = n - k - 1;
        const double *col = A + (size_t)(k + 1) * n + k;  // x_i = col[i * n]
        double part = 0.0;
        for (int i = 1 + tid; i < L; i += kTriThreads) {
            const double x = col[(size_t)i * n];
            part += x * x;
        }
        const double sigma = block_sum(part, red);
        const double x0 = col[0];
        double beta = x0, t = 0.0, scale = 0.0;
        if (sigma != 0.0) {
            const double mu = sqrt(x0 * x0 + sigma);
            beta = x0 >= 0.0 ? -mu : mu;
            t = (beta - x0) / beta;
            scale = 1.0 / (x0 - beta);
        }
        for (int i = tid; i < L; i += kTriThreads) v[i] = i == 0 ? 1.0 : (t != 0.0 ? col[(size_t)i * n] * scale : 0.0);
        __syncthreads();
        if (blockIdx.x == 0) {
            if (tid == 0) {
                d[k] = A[(size_t)k * n + k];
                e[k] = beta;
                tau[k] = t;
            }
            for (int i = tid; i < L; i += kTriThreads) Vh[(size_t)k * n + k + 1 + i] = v[i];
        }
        if (t != 0.0) {
            // p = t A22 v, one warp per row
            for (int r = gwarp; r < L; r += nwarps) {
                const double *row = A + (size_t)(k + 1 + r) * n + k + 1;
                double s = 0.0;
                for (int j = lane; j < L; j += 32) s += row[j] * v[j];
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) p[r] = t * s;
            }
            grid.sync();
            double pv = 0.0;
            for (int i = tid; i < L; i += kTriThreads) pv += p[i] * v[i];
            const double K = 0.5 * t * block_sum(pv, red);
            for (int i = tid; i < L; i += kTriThreads) w[i] = p[i] - K * v[i];
            __syncthreads();
            // A22 -= v w^T + w v^T, one warp per row
            for (int r = gwarp; r < L; r += nwarps) {
                double *row = A + (size_t)(k + 1 + r) * n + k + 1;
                const double vr = v[r], wr = w[r];
                for (int j = lane; j < L; j += 32) row[j] -= vr * w[j] + wr * v[j];
            }
        }
        grid.sync();
    }
    if (blockIdx.x == 0 && tid == 0) {
        d[n - 1] = A[(size_t)(n - 1) * n + (n - 1)];
        tau[n - 1] = 0.0;
    }
}

// Threads of k_tridiag_rows: one warp per SM sub-partition.  FP64 issues at a
// 64th of the FP32 rate here, so every FP64 instruction that all warps repeat
// (reductions, the reflector's scalars) costs its full issue time once per
// warp on a sub-partition; with one warp each that cost is paid once.
constexpr int kTrdThreads = 128;

// sum over the block (kTrdThreads threads); result in all threads
__device__ __forceinline__ double block_sum128(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();  // red may still be read from the previous call
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    return (red[0] + red[1]) + (red[2] + red[3]);
}

// Sums over the 32 lanes of RMAX values per lane by halving: at the step with
// offset o every lane keeps the half of its values selected by its lane bit o
// and adds the partner's copy of that half, so the adds per lane are RMAX - 1
// plus log2(32 / RMAX) instead of 5 RMAX.  Afterwards lane l holds the total
// of value l / (32 / RMAX).
template <int RMAX>
__device__ __forceinline__ double warp_sum_rows(double (&a)[RMAX], int lane) {
    int off = 16;
#pragma unroll
    for (int h = RMAX / 2; h >= 1; h /= 2) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double keep = up ? a[i + h] : a[i];
            const double send = up ? a[i] : a[i + h];
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
        off >>= 1;
    }
    double s = a[0];
    for (; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return s;
}

// Tridiagonalisation with the matrix resident in shared memory.  CTA b owns
// the rows b, b + G, b + 2G, ... (full length n), so the product p = t A22 v
// and the rank-2 update of every column read and write only shared memory,
// and one grid barrier per column suffices: before it every CTA writes its
// entries of p, and the owner of row k+1 writes that row as it stands before
// the update of column k; after it every CTA forms w and, from that row, the
// updated row k+1, which by symmetry is the next column to reduce.  The update
// of column k is applied to the owned rows in the same pass as the product of
// column k+1.  The arithmetic per column is that of k_tridiag.
// Shared memory: R n (owned rows, R = ceil(n / G) <= RMAX) + 4 n doubles.
template <int RMAX>
__global__ void __launch_bounds__(kTrdThreads) k_tridiag_rows(int n, const double *__restrict__ A, double *__restrict__ d,
                                                            double *__restrict__ e, double *__restrict__ tau,
                                                            double *__restrict__ Vh, double *__restrict__ pbuf,
                                                            double *__restrict__ rbuf) {
    constexpr int NW = kTrdThreads / 32;
    cg::grid_group grid = cg::this_grid();
    extern __shared__ double sm[];
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int R = (n - b + G - 1) / G;          // rows owned by this CTA
    const int Rmax = (n + G - 1) / G;
    double *rows = sm;                           // Rmax x n
    double *xs = rows + (size_t)Rmax * n;        // row k: xs[i] = A[k, k + i]
    double *v = xs + n, *vp = v + n, *w = vp + n;  // reflector of column k, of column k - 1; w of column k - 1
    __shared__ double red[NW];
    __shared__ double redr[NW][RMAX];
    for (int i = 0; i < R; ++i) {
        const double *src = A + (size_t)(b + i * G) * n;
        for (int j = tid; j < n; j += kTrdThreads) rows[(size_t)i * n + j] = src[j];
    }
    for (int j = tid; j < n; j += kTrdThreads) xs[j] = A[j];
    __syncthreads();
    for (int k = 0; k + 1 < n; ++k) {
        const int L = n - k - 1;
        // reflector of y = xs[1 .. L] (column k below the diagonal)
        double part = 0.0;
        for (int i = 1 + tid; i < L; i += kTrdThreads) part = fma(xs[1 + i], xs[1 + i], part);
        const double sigma = block_sum128(part, red);
        const double x0 = xs[1];
        double beta = x0, t = 0.0, scale = 0.0;
        if (sigma != 0.0) {
            const double mu = sqrt(fma(x0, x0, sigma));
            beta = x0 >= 0.0 ? -mu : mu;
            // t = (beta - x0) / beta and scale = 1 / (x0 - beta) from one division
            const double dlt = x0 - beta, inv = 1.0 / (beta * dlt);
            t = -dlt * dlt * inv;
            scale = beta * inv;
        }
        for (int i = tid; i < L; i += kTrdThreads) {
            const double vi = i == 0 ? 1.0 : xs[1 + i] * scale;
            v[i] = vi;
            if (b == 0) Vh[(size_t)k * n + k + 1 + i] = vi;
        }
        if (b == 0 && tid == 0) {
            d[k] = xs[0];
            e[k] = beta;
            tau[k] = t;
        }
        __syncthreads();
        // owned rows r >= k + 1: update of column k - 1 (vectors vp, w, index
        // 0 <-> row k) on columns >= k + 1, then the product with v
        const int i0 = k + 1 > b ? (k + 1 - b + G - 1) / G : 0;
        double acc[RMAX];
#pragma unroll
        for (int i = 0; i < RMAX; ++i) acc[i] = 0.0;
        double *rb = rbuf + (size_t)(k & 1) * n;
        for (int j = tid; j < L; j += kTrdThreads) {
            const double vj = v[j];
            const double vpj = k > 0 ? vp[j + 1] : 0.0, wpj = k > 0 ? w[j + 1] : 0.0;
#pragma unroll
            for (int i = 0; i < RMAX; ++i) {
                if (i < i0 || i >= R) continue;
                const int r = b + i * G;
                double *a = rows + (size_t)i * n + k + 1 + j;
                double x = *a;
                if (k > 0) x -= vp[r - k] * wpj + w[r - k] * vpj;
                *a = x;
                acc[i] = fma(x, vj, acc[i]);
                if (r == k + 1) rb[j] = x;
            }
        }
        const double rs = warp_sum_rows<RMAX>(acc, lane);
        if ((lane & (32 / RMAX - 1)) == 0) redr[wid][lane / (32 / RMAX)] = rs;
        __syncthreads();
        if (tid >= i0 && tid < R) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < NW; ++q) s += redr[q][tid];
            pbuf[(size_t)(k & 1) * n + (b + tid * G - k - 1)] = t * s;
        }
        grid.sync();
        // w = p - (t/2)(p.v) v, then row k + 1 after the update of column k
        const double *pb = pbuf + (size_t)(k & 1) * n;
        double pv = 0.0;
        for (int j = tid; j < L; j += kTrdThreads) {
            const double pj = __ldcg(pb + j);
            xs[j] = __ldcg(rb + j);
            w[j] = pj;
            pv = fma(pj, v[j], pv);
        }
        const double K = 0.5 * t * block_sum128(pv, red);
        for (int j = tid; j < L; j += kTrdThreads) w[j] -= K * v[j];
        __syncthreads();
        const double w0 = w[0];
        for (int j = tid; j < L; j += kTrdThreads) xs[j] -= v[0] * w[j] + w0 * v[j];
        double *tmp = vp;
        vp = v;
        v = tmp;
        __syncthreads();
    }
    if (b == 0 && tid == 0) {
        d[n - 1] = xs[0];
        tau[n - 1] = 0.0;
    }
}

// Back transformation X = Q Z with Q = H_0 H_1 ... H_{n-2}: one warp per
// vector, its entries j = lane + 32 c in registers (n <= 32 C); the reflector
// of the next step is loaded into registers while the current one is applied
// and then stored to the other shared-memory buffer (one barrier per step).
template <int C>
__global__ void __launch_bounds__(256) k_tri_back_warp(int n, int m, const double *__restrict__ Vh,
                                                     const double *__restrict__ tau, const double *__restrict__ Z,
                                                     double *__restrict__ X, int ldx) {
    __shared__ double vs[2][32 * C];
    const int lane = threadIdx.x & 31, nthr = blockDim.x;
    const int i = blockIdx.x * (nthr >> 5) + (threadIdx.x >> 5);
    constexpr int P = (32 * C + 127) / 128;  // staged entries per thread (blockDim >= 128)
    double z[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int j = lane + 32 * c;
        z[c] = (i < m && j < n) ? Z[(size_t)i * n + j] : 0.0;
    }
    // reflector k: entries j > k of row k of Vh, zero elsewhere
    for (int j = threadIdx.x; j < 32 * C; j += nthr) vs[0][j] = (j > n - 2 && j < n) ? Vh[(size_t)(n - 2) * n + j] : 0.0;
    __syncthreads();
    int cur = 0;
    for (int k = n - 2; k >= 0; --k) {
        double pre[P];
        const bool more = k > 0;
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int j = threadIdx.x + q * nthr;
            pre[q] = (more && j < n && j > k - 1 && j < 32 * C) ? Vh[(size_t)(k - 1) * n + j] : 0.0;
        }
        const double t = tau[k];
        if (t != 0.0) {
            const double *vk = vs[cur];
            const int c0 = (k + 1) >> 5;  // entries below k + 1 are zero
            double s = 0.0;
#pragma unroll
            for (int c = 0; c < C; ++c)
                if (c >= c0) s += vk[lane + 32 * c] * z[c];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            s *= t;
#pragma unroll
            for (int c = 0; c < C; ++c)
                if (c >= c0) z[c] -= s * vk[lane + 32 * c];
        }
#pragma unroll
        for (int q = 0; q < P; ++q) {
            const int j = threadIdx.x + q * nthr;
            if (j < 32 * C) vs[cur ^ 1][j] = pre[q];
        }
        cur ^= 1;
        __syncthreads();
    }
    if (i < m) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const int j = lane + 32 * c;
            if (j < n) X[(size_t)j * ldx + i] = z[c];
        }
    }
}

// number of eigenvalues of T below x (Sturm sequence of the LDL^T of T - x I)
__device__ __forceinline__ int sturm_count(int n, const double *__restrict__ d, const double *__restrict__ e2,
                                           double x, double pivmin) {
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    int c = q < 0.0;
    for (int j = 1; j < n; ++j) {
        q = d[j] - x - e2[j - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        c += q < 0.0;
    }
    return c;
}

// e2[j] = e[j]^2, and the Gershgorin interval and ||T|| in bounds[0..2]
__global__ void k_tri_prep(int n, const double *__restrict__ d, const double *__restrict__ e, double *__restrict__ e2,
                           double *__restrict__ bounds, float *__restrict__ d32, float *__restrict__ e232) {
    __shared__ double red[3][kTriThreads / 32];
    double lo = DBL_MAX, hi = -DBL_MAX, nm = 0.0, e2max = 0.0;
    for (int j = threadIdx.x; j < n; j += kTriThreads) {
        const double r = (j > 0 ? fabs(e[j - 1]) : 0.0) + (j + 1 < n ? fabs(e[j]) : 0.0);
        lo = fmin(lo, d[j] - r);
        hi = fmax(hi, d[j] + r);
        nm = fmax(nm, fabs(d[j]) + r);
        d32[j] = (float)d[j];
        if (j + 1 < n) {
            e2[j] = e[j] * e[j];
            e232[j] = (float)e2[j];
            e2max = fmax(e2max, e2[j]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        nm = fmax(nm, __shfl_xor_sync(0xffffffffu, nm, o));
        e2max = fmax(e2max, __shfl_xor_sync(0xffffffffu, e2max, o));
    }
    __shared__ double red4[kTriThreads / 32];
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = lo;
        red[1][w] = hi;
        red[2][w] = nm;
        red4[w] = e2max;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kTriThreads / 32; ++i) {
            lo = fmin(lo, red[0][i]);
            hi = fmax(hi, red[1][i]);
            nm = fmax(nm, red[2][i]);
            e2max = fmax(e2max, red4[i]);
        }
        lo = fmin(lo, red[0][0]);
        hi = fmax(hi, red[1][0]);
        nm = fmax(nm, red[2][0]);
        e2max = fmax(e2max, red4[0]);
        const double pivmin = fmax(e2max, 1.0) * DBL_MIN / DBL_EPSILON;
        const double pad = 2.0 * DBL_EPSILON * nm + pivmin;
        bounds[0] = lo - pad;
        bounds[1] = hi + pad;
        bounds[2] = nm;
        bounds[3] = pivmin;
    }
}

__device__ __forceinline__ int sturm_count32(int n, const float *__restrict__ d, const float *__restrict__ e2, float x,
                                             float pivmin) {
    float q = d[0] - x;
    if (fabsf(q) < pivmin) q = -pivmin;
    int c = q < 0.f;
    for (int j = 1; j < n; ++j) {
        q = d[j] - x - e2[j - 1] / q;
        if (fabsf(q) < pivmin) q = -pivmin;
        c += q < 0.f;
    }
    return c;
}

// lambda_i, i < m: G eigenvalues per warp, L = 32 / G lanes each (L >= 2),
// multisection with L interior points (the bracket shrinks (L + 1)-fold per
// round).  FP32 rounds first (the FP32 pipe is ~60x the FP64 pipe) down to
// 1e-5 ||T||, then the bracket is checked with FP64 counts and widened until
// it holds, then FP64 rounds to full precision.  The FP64 rounds dominate; FP64
// issues at about one warp instruction per 64 cycles per SM sub-partition, so
// the launch gives each sub-partition about one warp, with G = ceil(m / (4 SMs)):
// fewer points per eigenvalue cost more rounds, a second warp on a
// sub-partition doubles every round.
__device__ __forceinline__ int group_le(bool le, int gbase, int L) {
    const unsigned bal = __ballot_sync(0xffffffffu, le);
    const unsigned g = (L == 32) ? bal : (bal >> gbase) & ((1u << L) - 1u);
    // lanes 0..j-1 of the group have count <= i (monotone up to rounding): take the highest
    return g == 0 ? 0 : 32 - __clz(g);
}

__global__ void k_tri_bisect(int n, int m, int G, const double *__restrict__ d, const double *__restrict__ e2,
                             const float *__restrict__ d32, const float *__restrict__ e232,
                             const double *__restrict__ bounds, double *__restrict__ lam) {
    const int lane = threadIdx.x & 31, warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int L = 32 / G, gi = lane / L, li = lane % L, gbase = gi * L;
    const int i = warp * G + gi;
    const bool valid = gi < G && i < m;
    if (warp * G >= m) return;  // uniform per warp
    const double glo = bounds[0], ghi = bounds[1], tn = bounds[2], pivmin = bounds[3];
    const double sect = 1.0 / (L + 1);
    double lo = glo, hi = ghi;
    // FP32 multisection
    const float pivmin32 = fmaxf((float)fmin(pivmin / DBL_MIN * FLT_MIN, 1e30), FLT_MIN / FLT_EPSILON);
    for (int round = 0; round < 64; ++round) {
        const bool go = valid && hi - lo > 1e-5 * tn;
        if (!__any_sync(0xffffffffu, go)) break;
        const double x = lo + (hi - lo) * ((li + 1) * sect);
        const bool le = go && sturm_count32(n, d32, e232, (float)x, pivmin32) <= i;
        const int nle = group_le(le, gbase, L);
        if (go) {
            const double nlo = nle > 0 ? lo + (hi - lo) * (nle * sect) : lo;
            const double nhi = nle < L ? lo + (hi - lo) * ((nle + 1) * sect) : hi;
            lo = nlo;
            hi = nhi;
        }
    }
    // FP64 check: count(lo) <= i < count(hi), widen otherwise
    double w = fmax(hi - lo, 1e-5 * tn);
    bool checked = !valid;
    for (int t = 0; t < 64; ++t) {
        if (!__any_sync(0xffffffffu, !checked)) break;
        const double x = li == 0 ? lo : hi;
        const int c = (!checked && li < 2) ? sturm_count(n, d, e2, x, pivmin) : 0;
        const int clo = __shfl_sync(0xffffffffu, c, gbase), chi = __shfl_sync(0xffffffffu, c, gbase + 1);
        if (!checked) {
            const bool okl = clo <= i || lo <= glo, okh = chi > i || hi >= ghi;
            if (okl && okh) {
                checked = true;
            } else {
                if (!okl) lo = fmax(glo, lo - w);
                if (!okh) hi = fmin(ghi, hi + w);
                w *= 2.0;
            }
        }
    }
    // FP64 multisection to 2 eps max(|lambda|, ||T||): the absolute accuracy
    // of a dense symmetric eigensolve (a relative stop alone would drive the
    // bracket of an eigenvalue at zero down to pivmin)
    const double atol = 2.0 * DBL_EPSILON * tn + pivmin;
    for (int round = 0; round < 200; ++round) {
        const double mid = 0.5 * (lo + hi);
        const bool go = valid && !(hi - lo <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) + atol || mid == lo ||
                                   mid == hi);
        if (!__any_sync(0xffffffffu, go)) break;
        const double x = lo + (hi - lo) * ((li + 1) * sect);
        const bool le = go && sturm_count(n, d, e2, x, pivmin) <= i;
        const int nle = group_le(le, gbase, L);
        if (go) {
            const double nlo = nle > 0 ? lo + (hi - lo) * (nle * sect) : lo;
            const double nhi = nle < L ? lo + (hi - lo) * ((nle + 1) * sect) : hi;
            lo = nlo;
            hi = nhi;
        }
    }
    if (valid && li == 0) lam[i] = 0.5 * (lo + hi);
}

// uniform in [-1, 1) from a 64-bit hash (splitmix64 finaliser)
__device__ __forceinline__ double hash_uniform(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// inverse iteration, one warp per cluster [cstart[c], cstart[c + 1]); Z is m x n
// (vector-major); LU scratch: 5 n doubles + n flags per cluster
__global__ void k_tri_invit(int n, const double *__restrict__ d, const double *__restrict__ e,
                            const double *__restrict__ bounds, const double *__restrict__ lam,
                            const int *__restrict__ cstart, double *__restrict__ Z, double *__restrict__ scratch,
                            unsigned char *__restrict__ pivflag) {
    const int c = blockIdx.x, lane = threadIdx.x;
    const int i0 = cstart[c], i1 = cstart[c + 1];
    double *u0i = scratch + (size_t)c * 5 * n;  // reciprocal of the pivot
    double *u1 = u0i + n, *u2 = u1 + n, *l = u2 + n, *y = l + n;
    unsigned char *piv = pivflag + (size_t)c * n;
    const double small = DBL_EPSILON * fmax(bounds[2], DBL_MIN);
    for (int i = i0; i < i1; ++i) {
        double *z = Z + (size_t)i * n;
        const double lmb = lam[i];
        if (lane == 0) {
            // T - lmb I = P L U, U with three diagonals (u0, u1, u2)
            double cd = d[0] - lmb, cu = n > 1 ? e[0] : 0.0;
            for (int j = 0; j + 1 < n; ++j) {
                const double nd = d[j + 1] - lmb, nu = j + 2 < n ? e[j + 1] : 0.0, sub = e[j];
                if (fabs(cd) >= fabs(sub)) {
                    piv[j] = 0;
                    if (fabs(cd) < small) cd = cd >= 0.0 ? small : -small;
                    const double lj = sub / cd;
                    l[j] = lj;
                    u0i[j] = 1.0 / cd;
                    u1[j] = cu;
                    u2[j] = 0.0;
                    cd = nd - lj * cu;
                    cu = nu;
                } else {
                    piv[j] = 1;
                    const double lj = cd / sub;
                    l[j] = lj;
                    u0i[j] = 1.0 / sub;
                    u1[j] = nd;
                    u2[j] = nu;
                    cd = cu - lj * nd;
                    cu = -lj * nu;
                }
            }
            if (fabs(cd) < small) cd = cd >= 0.0 ? small : -small;
            u0i[n - 1] = 1.0 / cd;
        }
        for (int j = lane; j < n; j += 32) z[j] = hash_uniform(((uint64_t)i << 32) ^ (uint64_t)j);
        __syncwarp();
        for (int it = 0; it < 3; ++it) {
            if (lane == 0) {
                for (int j = 0; j < n; ++j) y[j] = z[j];
                for (int j = 0; j + 1 < n; ++j) {
                    if (piv[j]) {
                        const double t = y[j];
                        y[j] = y[j + 1];
                        y[j + 1] = t;
                    }
                    y[j + 1] -= l[j] * y[j];
                }
                double z1 = 0.0, z2 = 0.0;  // z[j + 1], z[j + 2]
                for (int j = n - 1; j >= 0; --j) {
                    double s = y[j];
                    if (j + 1 < n) s -= u1[j] * z1;
                    if (j + 2 < n) s -= u2[j] * z2;
                    const double zj = s * u0i[j];
                    z[j] = zj;
                    z2 = z1;
                    z1 = zj;
                }
            }
            __syncwarp();
            // orthogonal to the earlier vectors of the cluster, then unit length
            for (int jv = i0; jv < i; ++jv) {
                const double *o = Z + (size_t)jv * n;
                double s = 0.0;
                for (int j = lane; j < n; j += 32) s += o[j] * z[j];
                s = warp_sum(s);
                for (int j = lane; j < n; j += 32) z[j] -= s * o[j];
                __syncwarp();
            }
            double s = 0.0;
            for (int j = lane; j < n; j += 32) s += z[j] * z[j];
            s = warp_sum(s);
            const double inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
            for (int j = lane; j < n; j += 32) z[j] *= inv;
            __syncwarp();
        }
    }
}

// X[:, i] = Q z_i for i in this CTA's group; vectors kept in shared memory
__global__ void __launch_bounds__(kTriThreads) k_tri_back(int n, int m, int per_cta, const double *__restrict__ Vh,
                                                        const double *__restrict__ tau, const double *__restrict__ Z,
                                                        double *__restrict__ X, int ldx) {
    extern __shared__ double zs[];  // per_cta x n
    __shared__ double red[kTriThreads / 32][8];
    __shared__ double dots[8];
    const int i0 = blockIdx.x * per_cta;
    const int cnt = min(per_cta, m - i0);
    for (int idx = threadIdx.x; idx < cnt * n; idx += kTriThreads) zs[idx] = Z[(size_t)i0 * n + idx];
    __syncthreads();
    for (int k = n - 2; k >= 0; --k) {
        const double t = tau[k];
        if (t == 0.0) continue;  // uniform across the CTA
        const double *v = Vh + (size_t)k * n;
        double part[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) part[c] = 0.0;
        for (int j = k + 1 + threadIdx.x; j < n; j += kTriThreads) {
            const double vj = v[j];
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c < cnt) part[c] += vj * zs[c * n + j];
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            double s = part[c];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            part[c] = s;
        }
        if ((threadIdx.x & 31) == 0)
#pragma unroll
            for (int c = 0; c < 8; ++c) red[threadIdx.x >> 5][c] = part[c];
        __syncthreads();
        if (threadIdx.x < 8) {
            double s = 0.0;
            for (int wi = 0; wi < kTriThreads / 32; ++wi) s += red[wi][threadIdx.x];
            dots[threadIdx.x] = t * s;
        }
        __syncthreads();
        for (int j = k + 1 + threadIdx.x; j < n; j += kTriThreads) {
            const double vj = v[j];
            for (int c = 0; c < cnt; ++c) zs[c * n + j] -= dots[c] * vj;
        }
        __syncthreads();
    }
    for (int idx = threadIdx.x; idx < cnt * n; idx += kTriThreads) {
        const int c = idx / n, j = idx % n;
        X[(size_t)j * ldx + i0 + c] = zs[idx];
    }
}

}  // namespace

size_t sym_eig_work_size(int n, int m) {
    // d e tau p e2 bounds(8) | Vh n^2 | Z m n | lam m | LU 5 n m | pivots n m bytes | cluster starts m + 1 ints
    // | d, e^2 in FP32 (n each)
    return (size_t)5 * n + 8 + (size_t)n * n + (size_t)m * n + m + (size_t)5 * n * m + ((size_t)n * m + 7) / 8 +
           ((size_t)m + 2) / 2 + 16 + (size_t)n + 8 + (size_t)4 * n + 8;
}

namespace {

// grid of k_tridiag_rows for an n x n matrix: G CTAs owning ceil(n / G) rows
// each; 0 if the rows do not fit in shared memory
int rows_grid(int n, int sms, size_t *smem, int *rmax) {
    const int G = std::max(1, std::min(sms, (n + 3) / 4));
    const int R = (n + G - 1) / G;
    *smem = ((size_t)R * n + 4 * (size_t)n) * sizeof(double);
    *rmax = R <= 4 ? 4 : R <= 8 ? 8 : 16;
    return (R <= 16 && *smem <= kTriSmemMax) ? G : 0;
}

template <int RMAX>
bool launch_tridiag_rows(cudaStream_t s, int G, size_t smem, int sms, int n, const double *A, double *d, double *e,
                         double *tau, double *Vh, double *pbuf, double *rbuf) {
    HSIM_SMEM_LIMIT_ONCE(k_tridiag_rows<RMAX>, kTriSmemMax);
    int per_sm = 0;
    HSIM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag_rows<RMAX>, kTrdThreads, smem));
    if ((int64_t)per_sm * sms < G) return false;
    int nn = n;
    void *args[] = {&nn, &A, &d, &e, &tau, &Vh, &pbuf, &rbuf};
    HSIM_CUDA(cudaLaunchCooperativeKernel((void *)k_tridiag_rows<RMAX>, dim3(G), dim3(kTrdThreads), args, smem, s));
    HSIM_LAUNCHED();
    return true;
}

template <int C>
void launch_back_warp(cudaStream_t s, int warps, int n, int m, const double *Vh, const double *tau, const double *Z,
                      double *X, int ldx) {
    k_tri_back_warp<C><<<cdiv(m, warps), 32 * warps, 0, s>>>(n, m, Vh, tau, Z, X, ldx);
    HSIM_LAUNCHED();
}

}  // namespace

void sym_eig(cudaStream_t s, int n, int m, double *A, double *evals, double *X, int ldx, double *work) {
    HSIM_CHECK_ARG(n >= 1 && m >= 1 && m <= n, "sym_eig: bad sizes");
    double *d = work, *e = d + n, *tau = e + n, *p = tau + n, *e2 = p + n, *bounds = e2 + n;
    double *Vh = bounds + 8, *Z = Vh + (size_t)n * n, *lam = Z + (size_t)m * n, *lu = lam + m;
    unsigned char *pivf = reinterpret_cast<unsigned char *>(lu + (size_t)5 * n * m);
    int *cst = reinterpret_cast<int *>(reinterpret_cast<double *>(pivf) + ((size_t)n * m + 7) / 8);
    float *d32 = reinterpret_cast<float *>(reinterpret_cast<double *>(cst) + ((size_t)m + 2) / 2 + 8);
    float *e232 = d32 + n;
    double *pbuf = reinterpret_cast<double *>(e232 + n) + 4, *rbuf = pbuf + 2 * (size_t)n;
    if (n == 1) {
        HSIM_CUDA(cudaMemcpyAsync(evals, A, sizeof(double), cudaMemcpyDeviceToDevice, s));
        const double one = 1.0;
        HSIM_CUDA(cudaMemcpyAsync(X, &one, sizeof(double), cudaMemcpyHostToDevice, s));
        HSIM_CUDA(cudaStreamSynchronize(s));
        return;
    }
    int dev = 0, sms = 0;
    HSIM_CUDA(cudaGetDevice(&dev));
    HSIM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // HSIM_TRACE=2: stage times of every call
    static const bool detail = [] {
        const char *ev = std::getenv("HSIM_TRACE");
        return ev && std::atoi(ev) >= 2;
    }();
    cudaEvent_t t0 = nullptr, t1 = nullptr, t2 = nullptr, t3 = nullptr, t4 = nullptr;
    if (detail) {
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        cudaEventCreate(&t2);
        cudaEventCreate(&t3);
        cudaEventCreate(&t4);
        cudaEventRecord(t0, s);
    }
    // 1. tridiagonalisation: rows resident in shared memory (one grid barrier
    // per column) where they fit, else rows in global memory (two barriers)
    size_t rsmem = 0;
    int rmax = 0;
    const int G = rows_grid(n, sms, &rsmem, &rmax);
    bool done = false;
    if (G > 0) {
        if (rmax == 4) done = launch_tridiag_rows<4>(s, G, rsmem, sms, n, A, d, e, tau, Vh, pbuf, rbuf);
        else if (rmax == 8) done = launch_tridiag_rows<8>(s, G, rsmem, sms, n, A, d, e, tau, Vh, pbuf, rbuf);
        else done = launch_tridiag_rows<16>(s, G, rsmem, sms, n, A, d, e, tau, Vh, pbuf, rbuf);
    }
    if (!done) {
        const size_t smem = 2 * (size_t)n * sizeof(double);
        HSIM_CHECK_ARG(smem <= kTriSmemMax, "sym_eig: matrix too large for the tridiagonalisation kernel");
        HSIM_SMEM_LIMIT_ONCE(k_tridiag, kTriSmemMax);
        int per_sm = 0;
        HSIM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tridiag, kTriThreads, smem));
        HSIM_CHECK_ARG(per_sm >= 1, "sym_eig: tridiagonalisation kernel does not fit on an SM");
        const int grid = std::max(1, std::min(sms, (n + 7) / 8));
        int nn = n;
        void *args[] = {&nn, &A, &d, &e, &tau, &Vh, &p};
        HSIM_CUDA(cudaLaunchCooperativeKernel((void *)k_tridiag, dim3(grid), dim3(kTriThreads), args, smem, s));
        HSIM_LAUNCHED();
    }
    // 2. eigenvalues
    k_tri_prep<<<1, kTriThreads, 0, s>>>(n, d, e, e2, bounds, d32, e232);
    HSIM_LAUNCHED();
    if (detail) cudaEventRecord(t1, s);
    // about one warp per SM: G eigenvalues per warp (L = 32 / G >= 2 lanes each)
    // FP64 issues per SM sub-partition: about one warp on each of the 4 x SMs
    // sub-partitions (blocks of four warps, one per sub-partition)
    const int per_warp = std::max(1, std::min(16, (m + 4 * sms - 1) / (4 * sms)));
    const int nwarps = (m + per_warp - 1) / per_warp;
    k_tri_bisect<<<(nwarps + 3) / 4, 128, 0, s>>>(n, m, per_warp, d, e2, d32, e232, bounds, lam);
    HSIM_LAUNCHED();
    if (detail) cudaEventRecord(t2, s);
    // 3. clusters on the host, then inverse iteration
    std::vector<double> hl(m), hb(4);
    HSIM_CUDA(cudaMemcpyAsync(hl.data(), lam, m * sizeof(double), cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaMemcpyAsync(hb.data(), bounds, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaStreamSynchronize(s));
    std::vector<int> starts{0};
    for (int i = 1; i < m; ++i)
        if (hl[i] - hl[i - 1] > kClusterTol * hb[2]) starts.push_back(i);
    starts.push_back(m);
    const int nclusters = (int)starts.size() - 1;
    HSIM_CUDA(cudaMemcpyAsync(cst, starts.data(), starts.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    if (detail) cudaEventRecord(t2, s);
    k_tri_invit<<<nclusters, 32, 0, s>>>(n, d, e, bounds, lam, cst, Z, lu, pivf);
    HSIM_LAUNCHED();
    if (detail) cudaEventRecord(t3, s);
    // 4. back transformation: a warp per vector held in registers where n <=
    // 2048, else a few vectors per CTA in shared memory
    const int warps = std::max(4, std::min(8, (m + sms - 1) / sms));
    const int cw = (n + 31) / 32;
    if (cw <= 4) launch_back_warp<4>(s, warps, n, m, Vh, tau, Z, X, ldx);
    else if (cw <= 8) launch_back_warp<8>(s, warps, n, m, Vh, tau, Z, X, ldx);
    else if (cw <= 16) launch_back_warp<16>(s, warps, n, m, Vh, tau, Z, X, ldx);
    else if (cw <= 24) launch_back_warp<24>(s, warps, n, m, Vh, tau, Z, X, ldx);
    else if (cw <= 32) launch_back_warp<32>(s, warps, n, m, Vh, tau, Z, X, ldx);
    else if (cw <= 48) launch_back_warp<48>(s, warps, n, m, Vh, tau, Z, X, ldx);
    else if (cw <= 64) launch_back_warp<64>(s, warps, n, m, Vh, tau, Z, X, ldx);
    else {
        const int per_cta = std::max(1, std::min(8, (int)(kTriSmemMax / ((size_t)n * sizeof(double)))));
        const size_t bsm = (size_t)per_cta * n * sizeof(double);
        HSIM_SMEM_LIMIT_ONCE(k_tri_back, kTriSmemMax);
        k_tri_back<<<cdiv(m, per_cta), kTriThreads, bsm, s>>>(n, m, per_cta, Vh, tau, Z, X, ldx);
        HSIM_LAUNCHED();
    }
    HSIM_CUDA(cudaMemcpyAsync(evals, lam, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    // the host vector `starts` must outlive the copy above
    HSIM_CUDA(cudaStreamSynchronize(s));
    if (detail) {
        cudaEventRecord(t4, s);
        cudaEventSynchronize(t4);
        float a = 0, b = 0, c = 0, dd = 0;
        cudaEventElapsedTime(&a, t0, t1);
        cudaEventElapsedTime(&b, t1, t2);
        cudaEventElapsedTime(&c, t2, t3);
        cudaEventElapsedTime(&dd, t3, t4);
        int biggest = 0;
        for (size_t i = 0; i + 1 < starts.size(); ++i) biggest = std::max(biggest, starts[i + 1] - starts[i]);
        std::fprintf(stderr,
                     "[hsim] sym_eig n=%d m=%d tridiag %.2f ms eigenvalues %.2f ms vectors %.2f ms (%d clusters, "
                     "largest %d) back %.2f ms\n",
                     n, m, a, b, c, nclusters, biggest, dd);
        for (cudaEvent_t ev : {t0, t1, t2, t3, t4}) cudaEventDestroy(ev);
    }
}

}  // namespace k
}  // namespace hsim
