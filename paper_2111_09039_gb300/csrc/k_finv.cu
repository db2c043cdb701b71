// Inverted-factor form of the multifrontal LDL^T for the many-right-hand-side
// solves of the inverse iterations (Alg. 1, the solve with S - mu M).
//
// After the numeric factorisation front t holds, column-major nf x nf, the
// panel [L_ss; L_bs] (unit lower pivot block, rows of the ancestors) with D on
// the diagonal.  Walking the pivot block panel by panel makes the solves a
// chain of small dependent launches; instead every pivot block is inverted once
// per factorisation and the ancestor block multiplied by the inverse,
//     Linv = L_ss^-1   (unit lower, stored over L_ss; the diagonal keeps D)
//     W    = L_bs Linv (stored over L_bs),
// so that one tree height of the forward and of the backward substitution is
// one batched product each:
//     forward:  Y_s = Linv X_s,  X_b -= W X_s
//     backward: X_s = Linv^T D^-1 Y_s - W^T X_b
// (X_s: pivot rows of the front, contiguous; X_b: its ancestor rows).  The
// inversion doubles the block size per level,
//     [A 0; B C]^-1 = [A^-1 0; -C^-1 (B A^-1)  C^-1],
// starting from inverted 32 x 32 diagonal blocks; each level is two batched
// products over all fronts.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "common.h"
#include "kernels.h"

namespace hsim {
namespace k {

namespace {

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ---- inversion ---------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(32) k_inv_diag32(FrontDev fd, const int2 *__restrict__ blk, T *__restrict__ arena) {
    __shared__ T Ls[32][33];  // Ls[r][c] = L(b0 + r, b0 + c), r > c
    __shared__ T Xs[32][33];  // inverse, same indexing
    const int2 tb = blk[blockIdx.x];
    const int t = tb.x, b0 = tb.y;
    const int nf = fd.nf[t], ns = fd.ns[t];
    const int kb = min(32, ns - b0);
    T *F = arena + fd.foff[t];
    const int l = threadIdx.x;
    // lane l loads row l (coalesced along the column), then solves column l
    for (int c = 0; c < kb; ++c) Ls[l][c] = (l < kb && l > c) ? F[(int64_t)(b0 + c) * nf + b0 + l] : T(0);
    __syncwarp();
    if (l < kb) {
        Xs[l][l] = T(1);
        for (int r = l + 1; r < kb; ++r) {
            T s = Ls[r][l];
            for (int j = l + 1; j < r; ++j) s += Ls[r][j] * Xs[j][l];
            Xs[r][l] = -s;
        }
    }
    __syncwarp();
    for (int c = 0; c < kb; ++c)
        if (l < kb && l > c) F[(int64_t)(b0 + c) * nf + b0 + l] = Xs[l][c];
}

template <typename T>
__device__ __forceinline__ T tri_load(const T *p, int64_t idx, int i, int k, bool unit_lower) {
    if (!unit_lower) return p[idx];
    return i > k ? p[idx] : (i == k ? T(1) : T(0));
}

__device__ __forceinline__ int find_task(const GemmTask *tasks, int ntasks, int tile) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile0 <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_tasks(const GemmTask *__restrict__ tasks, int ntasks,
                                                    const T *__restrict__ Ab, const T *__restrict__ Bb,
                                                    T *__restrict__ Cb) {
    constexpr int BT = kGemmTile, BK = 16;
    __shared__ T As[BK][BT + 1];
    __shared__ T Bs[BK][BT + 1];
    const GemmTask tk = tasks[find_task(tasks, ntasks, blockIdx.x)];
    const int local = blockIdx.x - tk.tile0;
    const int ntn = (tk.N + BT - 1) / BT;
    const int m0 = (local / ntn) * BT, n0 = (local % ntn) * BT;
    const bool ua = tk.flags & kGemmAUnitLower, ub = tk.flags & kGemmBUnitLower;
    const T *A = Ab + tk.a, *B = Bb + tk.b;
    T *C = Cb + tk.c;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // tx: rows, ty: columns
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
    // a unit lower A has A(i, k) = 0 for k > i; a unit lower B has B(k, j) = 0 for k < j
    const int kbeg = ub ? (n0 / BK) * BK : 0;
    const int kend = ua ? min(tk.K, m0 + BT) : tk.K;
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        for (int idx = threadIdx.x; idx < BK * BT; idx += 256) {
            const int i = idx % BT, kk = idx / BT;
            const int gi = m0 + i, gk = k0 + kk;
            As[kk][i] = (gi < tk.M && gk < tk.K) ? tri_load(A, (int64_t)gk * tk.lda + gi, gi, gk, ua) : T(0);
        }
        for (int idx = threadIdx.x; idx < BK * BT; idx += 256) {
            const int kk = idx % BK, j = idx / BK;
            const int gk = k0 + kk, gj = n0 + j;
            Bs[kk][j] = (gk < tk.K && gj < tk.N) ? tri_load(B, (int64_t)gj * tk.ldb + gk, gk, gj, ub) : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[kk][tx + 16 * u];
                b[u] = Bs[kk][ty + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
        __syncthreads();
    }
    const T sg = (tk.flags & kGemmNeg) ? T(-1) : T(1);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = m0 + tx + 16 * u;
        if (i >= tk.M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int j = n0 + ty + 16 * v;
            if (j < tk.N) C[(int64_t)j * tk.ldc + i] = sg * acc[u][v];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_copy_tasks(const GemmTask *__restrict__ tasks, int ntasks,
                                                    const T *__restrict__ Ab, T *__restrict__ Cb) {
    constexpr int BT = kGemmTile;
    const GemmTask tk = tasks[find_task(tasks, ntasks, blockIdx.x)];
    const int local = blockIdx.x - tk.tile0;
    const int ntn = (tk.N + BT - 1) / BT;
    const int m0 = (local / ntn) * BT, n0 = (local % ntn) * BT;
    for (int idx = threadIdx.x; idx < BT * BT; idx += 256) {
        const int i = m0 + idx % BT, j = n0 + idx / BT;
        if (i < tk.M && j < tk.N) Cb[tk.c + (int64_t)j * tk.ldc + i] = Ab[tk.a + (int64_t)j * tk.lda + i];
    }
}

template <typename T>
__global__ void k_reciprocal(int n, const T *__restrict__ x, T *__restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = T(1) / x[i];
}

// ---- solves ---------------------------------------------------------------

// four consecutive values of row `row` from column c (zero past k or for an
// invalid row)
template <typename T>
__device__ __forceinline__ void load4(T (&d)[4], const T *X, int64_t row, bool ok, int c, int k, int ldx, bool vec) {
    const T *p = X + row * ldx + c;
    if (ok && vec && c + 4 <= k) {
        if constexpr (sizeof(T) == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(p);
            d[0] = v.x, d[1] = v.y, d[2] = v.z, d[3] = v.w;
        } else {
            const double2 v0 = reinterpret_cast<const double2 *>(p)[0], v1 = reinterpret_cast<const double2 *>(p)[1];
            d[0] = v0.x, d[1] = v0.y, d[2] = v1.x, d[3] = v1.y;
        }
    } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) d[v] = (ok && c + v < k) ? p[v] : T(0);
    }
}

template <typename T>
__device__ __forceinline__ void store4(T *p, const T (&a)[4], int avail, bool vec) {
    if (vec && avail >= 4) {
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(p) = make_float4(a[0], a[1], a[2], a[3]);
        } else {
            reinterpret_cast<double2 *>(p)[0] = make_double2(a[0], a[1]);
            reinterpret_cast<double2 *>(p)[1] = make_double2(a[2], a[3]);
        }
    } else {
#pragma unroll
        for (int v = 0; v < 4; ++v)
            if (v < avail) p[v] = a[v];
    }
}

__device__ __forceinline__ void sub4_atomic(float *x, const float (&a)[4], int avail, bool vec) {
    if (vec && avail >= 4) {
        atomicAdd(reinterpret_cast<float4 *>(x), make_float4(-a[0], -a[1], -a[2], -a[3]));
    } else {
        for (int v = 0; v < 4 && v < avail; ++v) atomicAdd(x + v, -a[v]);
    }
}

// four consecutive shared-memory values (16-byte aligned)
template <typename T>
__device__ __forceinline__ void sts4(T *p, const T (&b)[4]) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(b[0], b[1], b[2], b[3]);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(b[0], b[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(b[2], b[3]);
    }
}
template <typename T>
__device__ __forceinline__ void lds4(T (&b)[4], const T *p) {
    if constexpr (sizeof(T) == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        b[0] = v.x, b[1] = v.y, b[2] = v.z, b[3] = v.w;
    } else {
        const double2 v0 = reinterpret_cast<const double2 *>(p)[0], v1 = reinterpret_cast<const double2 *>(p)[1];
        b[0] = v0.x, b[1] = v0.y, b[2] = v1.x, b[3] = v1.y;
    }
}

template <typename T>
__host__ __device__ constexpr int inv_cols() { return sizeof(T) == 4 ? 128 : 64; }  // columns of a solve tile

// Both solve kernels: 256 threads, output tile BM x BN (BN = 128 FP32
// columns), K in steps of 32 through two shared-memory stages; the next
// step's operands are loaded into registers while the current one is
// multiplied, then stored to the other stage (one barrier per step).
constexpr int kInvBK = 32;
// Backward heights with fewer than kBwdSplitPerSM CTAs per SM split their K
// range into up to kBwdMaxSplit chunks (10^6-vertex level, 750 columns: 2, 4
// and 8 CTAs per SM measured 11.7, 11.4 and 11.1 ms of backward per solve
// against 12.0 ms unsplit; the whole mixed solve 1.707, 1.702 and 1.699 s
// against 1.724 s)
constexpr int kBwdSplitPerSM = 8, kBwdMaxSplit = 8;

template <typename T, int BM>
constexpr size_t fwd_inv_smem(int stages) { return (size_t)stages * kInvBK * (BM + inv_cols<T>()) * sizeof(T); }
template <typename T, int BM>
constexpr size_t bwd_inv_smem(int stages) { return (size_t)stages * kInvBK * (BM + 1 + inv_cols<T>()) * sizeof(T); }

// CTA (front of the height, BM-row tile of its nf rows, column tile): rows
// r < ns of the product go to Y (store), rows r >= ns to the ancestors' rows
// of X (atomic subtraction: siblings share them).
template <typename T, int BM, int STAGES>
__global__ void __launch_bounds__(256, STAGES == 1 ? 4 : 2) k_solve_fwd_inv(FrontDev fd, const int *__restrict__ nodes,
                                                                          int rt_per,
                                                       const T *__restrict__ arena, int k, T *__restrict__ X,
                                                       T *__restrict__ Y, int ldx, bool vec) {
    constexpr int BK = kInvBK, BN = inv_cols<T>();
    constexpr int CG = BN / 4, RGS = 256 / CG, RPT = BM / RGS;
    constexpr int AE = BK * BM / 256, BE = BK * CG / 256;  // per-thread loads of one step
    static_assert(BK * BM % 256 == 0 && BK * CG % 256 == 0, "tile");
    // stage-major [2][BK][BN + BM]: B first (16-byte rows), then A; launches
    // whose fronts all have ns <= BK (one step) allocate stage 0 only
    extern __shared__ __align__(16) unsigned char inv_smem[];
    T *const base = reinterpret_cast<T *>(inv_smem);
    constexpr int STAGE = BK * (BN + BM);
    const int t = nodes[blockIdx.x / rt_per];
    const int r0 = (blockIdx.x % rt_per) * BM;
    const int nf = fd.nf[t], ns = fd.ns[t], ps = fd.pstart[t];
    if (r0 >= nf || ns == 0) return;
    const int c0 = blockIdx.y * BN;
    const T *F = arena + fd.foff[t];
    const int tid = threadIdx.x, cg = (tid % CG) * 4, rg = tid / CG;
    T acc[RPT][4];
#pragma unroll
    for (int u = 0; u < RPT; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
    T ra[AE], rb[BE][4];
    auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < AE; ++q) {
            const int idx = tid + 256 * q, i = idx % BM, kk = idx / BM;
            const int r = r0 + i, j = k0 + kk;
            T a = T(0);
            if (r < nf && j < ns) a = (r >= ns || r > j) ? F[(int64_t)j * nf + r] : (r == j ? T(1) : T(0));
            ra[q] = a;
        }
#pragma unroll
        for (int q = 0; q < BE; ++q) {
            const int idx = tid + 256 * q, kk = idx / CG, c = (idx % CG) * 4;
            load4(rb[q], X, (int64_t)ps + k0 + kk, k0 + kk < ns, c0 + c, k, ldx, vec);
        }
    };
    auto store = [&](int st) {
        T *bs = base + st * STAGE, *as = bs + BK * BN;
#pragma unroll
        for (int q = 0; q < AE; ++q) {
            const int idx = tid + 256 * q;
            as[(idx / BM) * BM + idx % BM] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < BE; ++q) {
            const int idx = tid + 256 * q;
            sts4(bs + (idx / CG) * BN + (idx % CG) * 4, rb[q]);
        }
    };
    auto compute = [&](int st) {
        const T *bs = base + st * STAGE, *as = bs + BK * BN;
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
            T b[4], a[RPT];
            lds4(b, bs + kk * BN + cg);
#pragma unroll
            for (int u = 0; u < RPT; ++u) a[u] = as[kk * BM + rg * RPT + u];
#pragma unroll
            for (int u = 0; u < RPT; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
    };
    // Linv(r, j) = 0 for j > r: a tile inside the pivot rows stops at its last row
    const int kend = (r0 + BM <= ns) ? r0 + BM : ns;
    if constexpr (STAGES == 1) {
        for (int k0 = 0; k0 < kend; k0 += BK) {
            load(k0);
            store(0);
            __syncthreads();
            compute(0);
            __syncthreads();
        }
    } else {
        load(0);
        store(0);
        __syncthreads();
        for (int k0 = 0, st = 0; k0 < kend; k0 += BK, st ^= 1) {
            const bool more = k0 + BK < kend;
            if (more) load(k0 + BK);
            compute(st);
            if (more) store(st ^ 1);
            __syncthreads();
        }
    }
    const int *rows = fd.rows + fd.rows_off[t];
    const int avail = k - c0 - cg;
    if (avail <= 0) return;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int r = r0 + rg * RPT + u;
        if (r >= nf) continue;
        if (r < ns) store4(Y + (int64_t)(ps + r) * ldx + c0 + cg, acc[u], avail, vec);
        else sub4_atomic(X + (int64_t)rows[r] * ldx + c0 + cg, acc[u], avail, vec);
    }
}

// CTA (front of the height, BM-row tile of its ns pivot rows, column tile);
// K runs over the front's rows: pivots (Linv^T, Y scaled by D^-1), then the
// ancestors' rows (-W^T, final X rows gathered).
template <typename T, int BM, int STAGES>
__global__ void __launch_bounds__(256, STAGES == 1 ? 4 : 2) k_solve_bwd_inv(FrontDev fd, const int *__restrict__ nodes,
                                                                          int rt_per,
                                                       const T *__restrict__ arena, const T *__restrict__ dinv, int k,
                                                       T *__restrict__ X, const T *__restrict__ Y, int ldx, bool vec,
                                                       int ksplit) {
    constexpr int BK = kInvBK, BN = inv_cols<T>(), LDA = BM + 1;
    constexpr int CG = BN / 4, RGS = 256 / CG, RPT = BM / RGS;
    constexpr int AE = BK * BM / 256, BE = BK * CG / 256;
    static_assert(RPT >= 1 && BK * BM % 256 == 0 && BK * CG % 256 == 0, "tile");
    extern __shared__ __align__(16) unsigned char inv_smem[];
    T *Bs = reinterpret_cast<T *>(inv_smem);  // [STAGES][BK][BN] (16-byte aligned rows)
    T *As = Bs + STAGES * BK * BN;            // [STAGES][BK][BM + 1]
    const int t = nodes[blockIdx.x / rt_per];
    const int i0 = (blockIdx.x % rt_per) * BM;
    const int nf = fd.nf[t], ns = fd.ns[t], ps = fd.pstart[t];
    if (i0 >= ns) return;
    const int c0 = blockIdx.y * BN;
    const T *F = arena + fd.foff[t];
    const int *rows = fd.rows + fd.rows_off[t];
    const int tid = threadIdx.x, cg = (tid % CG) * 4, rg = tid / CG;
    T acc[RPT][4];
#pragma unroll
    for (int u = 0; u < RPT; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
    T ra[AE], rb[BE][4];
    auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < AE; ++q) {
            const int idx = tid + 256 * q, kk = idx % BK, ii = idx / BK;
            const int i = i0 + ii, r = k0 + kk;
            T a = T(0);
            if (i < ns && r < nf) {
                if (r >= ns) a = -F[(int64_t)i * nf + r];
                else a = r > i ? F[(int64_t)i * nf + r] : (r == i ? T(1) : T(0));
            }
            ra[q] = a;
        }
#pragma unroll
        for (int q = 0; q < BE; ++q) {
            const int idx = tid + 256 * q, kk = idx / CG, c = (idx % CG) * 4;
            const int r = k0 + kk;
            if (r < ns) {
                load4(rb[q], Y, (int64_t)ps + r, true, c0 + c, k, ldx, vec);
                const T di = dinv[ps + r];
#pragma unroll
                for (int v = 0; v < 4; ++v) rb[q][v] *= di;
            } else {
                load4(rb[q], X, r < nf ? (int64_t)rows[r] : 0, r < nf, c0 + c, k, ldx, vec);
            }
        }
    };
    auto store = [&](int st) {
        T *as = As + st * BK * LDA, *bs = Bs + st * BK * BN;
#pragma unroll
        for (int q = 0; q < AE; ++q) {
            const int idx = tid + 256 * q;
            as[(idx % BK) * LDA + idx / BK] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < BE; ++q) {
            const int idx = tid + 256 * q;
            sts4(bs + (idx / CG) * BN + (idx % CG) * 4, rb[q]);
        }
    };
    auto compute = [&](int st) {
        const T *as = As + st * BK * LDA, *bs = Bs + st * BK * BN;
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
            T b[4], a[RPT];
            lds4(b, bs + kk * BN + cg);
#pragma unroll
            for (int u = 0; u < RPT; ++u) a[u] = as[kk * LDA + rg * RPT + u];
#pragma unroll
            for (int u = 0; u < RPT; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
        }
    };
    // Linv^T(i, r) = Linv(r, i) = 0 for r < i: start at the tile's first row.
    // Split K: chunk blockIdx.z of ksplit chunks of whole BK steps (the
    // partial products are added into X, zeroed beforehand)
    const int kfirst = (i0 / BK) * BK, steps = (nf - kfirst + BK - 1) / BK, cs = (steps + ksplit - 1) / ksplit;
    const int kbeg = kfirst + (int)blockIdx.z * cs * BK, kend = min(nf, kbeg + cs * BK);
    if (kbeg >= nf) return;
    if constexpr (STAGES == 1) {
        for (int k0 = kbeg; k0 < kend; k0 += BK) {
            load(k0);
            store(0);
            __syncthreads();
            compute(0);
            __syncthreads();
        }
    } else {
        load(kbeg);
        store(0);
        __syncthreads();
        for (int k0 = kbeg, st = 0; k0 < kend; k0 += BK, st ^= 1) {
            const bool more = k0 + BK < kend;
            if (more) load(k0 + BK);
            compute(st);
            if (more) store(st ^ 1);
            __syncthreads();
        }
    }
    const int avail = k - c0 - cg;
    if (avail <= 0) return;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
        const int i = i0 + rg * RPT + u;
        if (i >= ns) continue;
        if constexpr (sizeof(T) == 4) {
            if (ksplit > 1) {
                T neg[4];
#pragma unroll
                for (int v = 0; v < 4; ++v) neg[v] = -acc[u][v];
                sub4_atomic(X + (int64_t)(ps + i) * ldx + c0 + cg, neg, avail, vec);
                continue;
            }
        }
        store4(X + (int64_t)(ps + i) * ldx + c0 + cg, acc[u], avail, vec);
    }
}

// X rows [pstart, pstart + ns) of the listed fronts set to zero (columns < k):
// CTA (front, y) takes rows y, y + gridDim.y, ...
template <typename T>
__global__ void k_zero_pivot_rows(FrontDev fd, const int *__restrict__ nodes, int k, T *__restrict__ X, int ldx) {
    const int t = nodes[blockIdx.x];
    const int ns = fd.ns[t], ps = fd.pstart[t];
    for (int r = blockIdx.y; r < ns; r += gridDim.y)
        for (int c = threadIdx.x; c < k; c += blockDim.x) X[(int64_t)(ps + r) * ldx + c] = T(0);
}

// ---- the lowest two tree heights fused ------------------------------------------
//
// A front P of height 1 and its children (all leaves) in one CTA per column
// tile of kFuseCols right-hand sides.  Shared memory holds P's nf_P rows and
// the children's pivot rows of the tile.  Forward: each child's product
// updates P's pivot rows in place and accumulates its updates of P's
// ancestor rows (the rows of P beyond its pivots, which a child's ancestor
// rows map into through relmap) as deltas; then P's product; the deltas
// reach X once, by atomic subtraction (siblings of P share those rows).  The
// forward stores D^-1 Y for these fronts (the product the backward reads;
// the same rounding as scaling in the backward).  Backward: P's pivot rows
// from D^-1 Y and P's ancestor rows, then each child's pivot rows from D^-1 Y
// and P's rows, all read from shared memory.  The products of the per-height
// kernels, summed in another order.
//
// Every global operand arrives by cp.async: the tile's rows at the start,
// each front's block (with its relmap and D^-1) while the previous front is
// multiplied (two buffers).  Each thread owns R rows x 4 columns of the
// output: R = 4 in the forward; in the backward, whose outputs are only the
// pivot rows (a few per front here), R = 1, 2 or 4, whichever leaves the
// longest row group shortest.  A front block is staged with its leading
// dimension padded to a multiple of four, so one shared load of R values
// gives the R rows' coefficients of a step, and the unit-triangular
// diagonal R x R blocks are masked in registers.
constexpr int kFuseCols = 64;
constexpr int kFuseCG = kFuseCols / 4, kFuseRG = 256 / kFuseCG;  // 16 column groups, 16 row groups
constexpr int kFuseMaxPiv = 4 * kFuseRG;                          // pivots of P at most (one pass)
constexpr int kFuseMaxAnc = 8 * kFuseRG;                          // ancestor rows of P at most
constexpr int kFuseMaxKids = 8;                                   // children of P at most

__host__ __device__ constexpr int pad4(int n) { return (n + 3) & ~3; }

// front buffer: the staged block, then relmap (ints), then D^-1 of the pivots
__host__ __device__ constexpr int fuse_block(int nf, int ns) {
    return pad4(ns * pad4(nf) > nf * pad4(ns) ? ns * pad4(nf) : nf * pad4(ns));
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src, int bytes) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// four values of row `row` from column c into shared memory (zero past k)
__device__ __forceinline__ void row4_async(float *dst, const float *X, int64_t row, int c, int k, int ldx, bool vec) {
    const float *p = X + row * ldx + c;
    if (vec) {
        const int n = k - c >= 4 ? 4 : (k - c > 0 ? k - c : 0);
        cp_async16(dst, n > 0 ? p : X, 4 * n);
    } else {
#pragma unroll
        for (int v = 0; v < 4; ++v) cp_async4(dst + v, c + v < k ? p + v : X, c + v < k ? 4 : 0);
    }
}

struct FuseMeta {
    int nf, ns, ps;
    int64_t foff, roff;
};

// the block of front m, its relmap and (forward) D^-1 of its pivots into buf;
// forward layout As[j * pad4(nf) + r] = F(r, j), backward At[r * pad4(ns) + i] = F(r, i)
template <bool FWD>
__device__ __forceinline__ void stage_front(const FuseMeta &m, const float *__restrict__ arena,
                                            const int *__restrict__ relmap, const float *__restrict__ dinv,
                                            float *buf) {
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const float *F = arena + m.foff;
    for (int j = warp; j < m.ns; j += 8)
        for (int r = lane; r < m.nf; r += 32) {
            float *d = FWD ? buf + (size_t)j * pad4(m.nf) + r : buf + (size_t)r * pad4(m.ns) + j;
            cp_async4(d, F + (size_t)j * m.nf + r, 4);
        }
    int *rel = reinterpret_cast<int *>(buf + fuse_block(m.nf, m.ns));
    for (int i = threadIdx.x; i < m.nf - m.ns; i += 256) cp_async4(rel + i, relmap + m.roff + i, 4);
    if (FWD) {
        float *ds = buf + fuse_block(m.nf, m.ns) + pad4(m.nf - m.ns);
        for (int i = threadIdx.x; i < m.ns; i += 256) cp_async4(ds + i, dinv + m.ps + i, 4);
    }
}

// R consecutive floats of shared memory (aligned to R floats)
template <int R>
__device__ __forceinline__ void lds_rows(float (&a)[R], const float *p) {
    if constexpr (R == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(p);
        a[0] = v.x, a[1] = v.y, a[2] = v.z, a[3] = v.w;
    } else if constexpr (R == 2) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        a[0] = v.x, a[1] = v.y;
    } else {
        a[0] = *p;
    }
}

// acc[u][v] += SIGN * sum_{j in [jb, je)} A[j * lda + r0 + u] * B(j)[c + v], u < R, B(j)
// the shared-memory row j of B, or row idx[j - ib] when idx is given
template <int SIGN, int R>
__device__ __forceinline__ void mac_rows(float (&acc)[R][4], const float *A, int lda, int r0, const float *B,
                                         const int *idx, int ib, int c, int jb, int je) {
#pragma unroll 4
    for (int j = jb; j < je; ++j) {
        float av[R];
        lds_rows<R>(av, A + (size_t)j * lda + r0);
        const int br = idx ? idx[j - ib] : j;
        const float4 b = *reinterpret_cast<const float4 *>(B + (size_t)br * kFuseCols + c);
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < R; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += (SIGN * av[u]) * bv[v];
    }
}

template <int R>
__device__ __forceinline__ void zero_rows(float (&acc)[R][4]) {
#pragma unroll
    for (int u = 0; u < R; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
}

__device__ __forceinline__ void add4(float *p, const float (&a)[4], float sg) {
    float4 d = *reinterpret_cast<float4 *>(p);
    d.x += sg * a[0];
    d.y += sg * a[1];
    d.z += sg * a[2];
    d.w += sg * a[3];
    *reinterpret_cast<float4 *>(p) = d;
}

// rows per thread for `rows` output rows over the 16 row groups: the fewest
// rows per thread in the longest group, four rows on ties (fewer shared loads
// per product)
__device__ __forceinline__ int pick_rows(int rows) {
    auto span = [&](int R) { return R * ((rows + R * kFuseRG - 1) / (R * kFuseRG)); };
    const int s4 = span(4), s2 = span(2), s1 = span(1);
    return s4 <= s2 && s4 <= s1 ? 4 : (s2 <= s1 ? 2 : 1);
}

// forward product of one staged front on rows r0..r0+R-1 (column-major As,
// unit lower triangle on the pivot rows): xs holds its pivot rows
template <int R>
__device__ __forceinline__ void fwd_rows(float (&acc)[R][4], const float *As, int nf, int ns, int r0, const float *xs,
                                         int cg) {
    zero_rows<R>(acc);
    const int lda = pad4(nf);
    mac_rows<1, R>(acc, As, lda, r0, xs, nullptr, 0, cg, 0, min(r0, ns));
    for (int j = r0; j < min(r0 + R, ns); ++j) {  // the diagonal block
        const float4 b = *reinterpret_cast<const float4 *>(xs + (size_t)j * kFuseCols + cg);
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int r = r0 + u;
            const float a = (r >= ns || r > j) ? As[(size_t)j * lda + r] : (r == j ? 1.f : 0.f);
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += a * bv[v];
        }
    }
}

// backward product of one staged front on outputs i0..i0+R-1 (row-major At):
// rows r < ns of B from xs (D^-1 Y), rows r >= ns from anc (row rel[r - ns]
// of anc when rel is given, else row r)
template <int R>
__device__ __forceinline__ void bwd_rows(float (&acc)[R][4], const float *At, int nf, int ns, int i0, const float *xs,
                                         const float *anc, const int *rel, int cg) {
    zero_rows<R>(acc);
    const int lda = pad4(ns), rd = min(i0 + R, ns);
    for (int r = i0; r < rd; ++r) {  // the diagonal block
        const float4 b = *reinterpret_cast<const float4 *>(xs + (size_t)r * kFuseCols + cg);
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int i = i0 + u;
            const float a = r > i ? At[(size_t)r * lda + i] : (r == i ? 1.f : 0.f);
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += a * bv[v];
        }
    }
    mac_rows<1, R>(acc, At, lda, i0, xs, nullptr, 0, cg, rd, ns);
    mac_rows<-1, R>(acc, At, lda, i0, anc, rel, ns, cg, ns, nf);
}

// the forward product of front m (a child of P, or P itself) and its outputs:
// pivot rows to Y (scaled by D^-1), the other rows into P's rows of Xs
template <int R>
__device__ __forceinline__ void fwd_front(const FuseMeta &m, const float *As, bool isP, int nsP, const float *xs,
                                          float *Xs, float *Y, int ldx, int c0, int cg, int rg, int avail, bool vec) {
    const int *rel = reinterpret_cast<const int *>(As + fuse_block(m.nf, m.ns));
    const float *ds = As + fuse_block(m.nf, m.ns) + pad4(m.nf - m.ns);
    for (int r0 = R * rg; r0 < m.nf; r0 += R * kFuseRG) {
        float acc[R][4];
        fwd_rows<R>(acc, As, m.nf, m.ns, r0, xs, cg);
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int r = r0 + u;
            if (r >= m.nf) break;
            if (r < m.ns) {
                const float di = ds[r];
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] *= di;
                if (avail > 0) store4(Y + (int64_t)(m.ps + r) * ldx + c0 + cg, acc[u], avail, vec);
            } else if (isP) {  // a delta of P's ancestor row r
                add4(Xs + (size_t)r * kFuseCols + cg, acc[u], 1.f);
            } else {           // P's row relmap(r): a pivot value, or a delta
                const int pr = rel[r - m.ns];
                add4(Xs + (size_t)pr * kFuseCols + cg, acc[u], pr < nsP ? -1.f : 1.f);
            }
        }
    }
}

// P's backward product (one pass: ns_P <= 16 R), then its pivot rows into Xs and X
template <int R>
__device__ __forceinline__ void bwd_parent(const FuseMeta &m, const float *At, float *Xs, float *X, int ldx, int c0,
                                           int cg, int rg, int avail, bool vec) {
    float acc[R][4];
    const int i0 = R * rg;
    if (i0 < m.ns) bwd_rows<R>(acc, At, m.nf, m.ns, i0, Xs, Xs, nullptr, cg);
    __syncthreads();
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int i = i0 + u;
        if (i >= m.ns) continue;
        sts4(Xs + (size_t)i * kFuseCols + cg, acc[u]);
        if (avail > 0) store4(X + (int64_t)(m.ps + i) * ldx + c0 + cg, acc[u], avail, vec);
    }
}

// a child's backward product: its pivot rows of X from xs (D^-1 Y) and P's rows
template <int R>
__device__ __forceinline__ void bwd_child(const FuseMeta &m, const float *At, const float *xs, const float *Xs,
                                          float *X, int ldx, int c0, int cg, int rg, int avail, bool vec) {
    const int *rel = reinterpret_cast<const int *>(At + fuse_block(m.nf, m.ns));
    for (int i0 = R * rg; i0 < m.ns; i0 += R * kFuseRG) {
        float acc[R][4];
        bwd_rows<R>(acc, At, m.nf, m.ns, i0, xs, Xs, rel, cg);
        if (avail <= 0) continue;
#pragma unroll
        for (int u = 0; u < R; ++u)
            if (i0 + u < m.ns) store4(X + (int64_t)(m.ps + i0 + u) * ldx + c0 + cg, acc[u], avail, vec);
    }
}

__device__ __forceinline__ void load_meta(FuseMeta *meta, const FrontDev &fd, int P, const int *child_ids, int cb,
                                          int nk, bool p_first) {
    const int t = threadIdx.x;
    if (t <= nk) {
        const int node = p_first ? (t == 0 ? P : child_ids[cb + t - 1]) : (t < nk ? child_ids[cb + t] : P);
        meta[t] = FuseMeta{fd.nf[node], fd.ns[node], fd.pstart[node], fd.foff[node], fd.relmap_off[node]};
    }
}

__global__ void __launch_bounds__(256, 3) k_solve_fwd_fused(FrontDev fd, const int *__restrict__ parents,
                                                         const int *__restrict__ child_ptr,
                                                         const int *__restrict__ child_ids,
                                                         const float *__restrict__ arena,
                                                         const float *__restrict__ dinv, int k, float *__restrict__ X,
                                                         float *__restrict__ Y, int ldx, int max_rows, int max_front,
                                                         bool vec) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ FuseMeta meta[kFuseMaxKids + 1];  // children, then P
    float *Xs = fsm;                                        // max_rows x kFuseCols
    float *const Fb = fsm + (size_t)max_rows * kFuseCols;  // two buffers of max_front floats
    const int P = parents[blockIdx.x];
    const int cb = child_ptr[blockIdx.x], nk = child_ptr[blockIdx.x + 1] - cb;
    load_meta(meta, fd, P, child_ids, cb, nk, false);
    __syncthreads();
    const int nfP = meta[nk].nf, nsP = meta[nk].ns, psP = meta[nk].ps;
    const int c0 = blockIdx.y * kFuseCols;
    const int tid = threadIdx.x, cg = (tid % kFuseCG) * 4, rg = tid / kFuseCG;
    const int avail = k - c0 - cg;
    // group 0: P's pivot rows, the children's pivot rows, the first block;
    // P's ancestor rows start as zero deltas
    for (int r = rg; r < nfP; r += kFuseRG) {
        float *d = Xs + (size_t)r * kFuseCols + cg;
        if (r < nsP) row4_async(d, X, (int64_t)psP + r, c0 + cg, k, ldx, vec);
        else *reinterpret_cast<float4 *>(d) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int t = 0, off = nfP; t < nk; off += meta[t].ns, ++t)
        for (int r = rg; r < meta[t].ns; r += kFuseRG)
            row4_async(Xs + (size_t)(off + r) * kFuseCols + cg, X, (int64_t)meta[t].ps + r, c0 + cg, k, ldx, vec);
    stage_front<true>(meta[0], arena, fd.relmap, dinv, Fb);
    cp_async_commit();
    if (nk >= 1) stage_front<true>(meta[1], arena, fd.relmap, dinv, Fb + max_front);
    cp_async_commit();
    for (int t = 0, off = nfP; t <= nk; ++t) {
        const FuseMeta m = meta[t];
        const float *As = Fb + (t & 1) * max_front;
        cp_async_wait<1>();
        __syncthreads();
        const bool isP = t == nk;
        const float *xs = isP ? Xs : Xs + (size_t)off * kFuseCols;
        // four rows per thread (fewer rows per thread measured slower here)
        fwd_front<4>(m, As, isP, nsP, xs, Xs, Y, ldx, c0, cg, rg, avail, vec);
        if (!isP) off += m.ns;
        __syncthreads();  // buffer t & 1 is free
        if (t + 2 <= nk) stage_front<true>(meta[t + 2], arena, fd.relmap, dinv, Fb + (t & 1) * max_front);
        cp_async_commit();
    }
    if (avail <= 0) return;
    const int *rowsP = fd.rows + fd.rows_off[P];
    for (int r = nsP + rg; r < nfP; r += kFuseRG) {
        float d[4];
        lds4(d, Xs + (size_t)r * kFuseCols + cg);
        sub4_atomic(X + (int64_t)rowsP[r] * ldx + c0 + cg, d, avail, vec);
    }
}

__global__ void __launch_bounds__(256, 3) k_solve_bwd_fused(FrontDev fd, const int *__restrict__ parents,
                                                         const int *__restrict__ child_ptr,
                                                         const int *__restrict__ child_ids,
                                                         const float *__restrict__ arena, int k, float *__restrict__ X,
                                                         const float *__restrict__ Y, int ldx, int max_rows,
                                                         int max_front, bool vec) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ FuseMeta meta[kFuseMaxKids + 1];  // P, then the children
    float *Xs = fsm;
    float *const Fb = fsm + (size_t)max_rows * kFuseCols;  // two buffers of max_front floats
    const int P = parents[blockIdx.x];
    const int cb = child_ptr[blockIdx.x], nk = child_ptr[blockIdx.x + 1] - cb;
    load_meta(meta, fd, P, child_ids, cb, nk, true);
    __syncthreads();
    const int nfP = meta[0].nf, nsP = meta[0].ns, psP = meta[0].ps;
    const int c0 = blockIdx.y * kFuseCols;
    const int tid = threadIdx.x, cg = (tid % kFuseCG) * 4, rg = tid / kFuseCG;
    const int avail = k - c0 - cg;
    const int *rowsP = fd.rows + fd.rows_off[P];
    // group 0: D^-1 Y of P's and the children's pivot rows (the forward
    // stored it), P's ancestor rows of X (final), P's block
    int anc[kFuseMaxAnc / kFuseRG];
#pragma unroll
    for (int q = 0; q < kFuseMaxAnc / kFuseRG; ++q) {
        const int r = nsP + rg + q * kFuseRG;
        anc[q] = r < nfP ? rowsP[r] : 0;
    }
    for (int r = rg; r < nsP; r += kFuseRG)
        row4_async(Xs + (size_t)r * kFuseCols + cg, Y, (int64_t)psP + r, c0 + cg, k, ldx, vec);
#pragma unroll
    for (int q = 0; q < kFuseMaxAnc / kFuseRG; ++q) {
        const int r = nsP + rg + q * kFuseRG;
        if (r < nfP) row4_async(Xs + (size_t)r * kFuseCols + cg, X, (int64_t)anc[q], c0 + cg, k, ldx, vec);
    }
    for (int t = 1, off = nfP; t <= nk; off += meta[t].ns, ++t)
        for (int r = rg; r < meta[t].ns; r += kFuseRG)
            row4_async(Xs + (size_t)(off + r) * kFuseCols + cg, Y, (int64_t)meta[t].ps + r, c0 + cg, k, ldx, vec);
    stage_front<false>(meta[0], arena, fd.relmap, nullptr, Fb);
    cp_async_commit();
    if (nk >= 1) stage_front<false>(meta[1], arena, fd.relmap, nullptr, Fb + max_front);
    cp_async_commit();
    for (int t = 0, off = nfP; t <= nk; ++t) {
        const FuseMeta m = meta[t];
        const float *At = Fb + (t & 1) * max_front;
        cp_async_wait<1>();
        __syncthreads();  // also: P's pivot rows of Xs written
        if (t == 0) {
            // X_P = Linv^T D^-1 Y_P - W^T X_anc in one pass (ns_P <= 64), then into Xs
            if (nsP <= kFuseRG) bwd_parent<1>(m, At, Xs, X, ldx, c0, cg, rg, avail, vec);
            else if (nsP <= 2 * kFuseRG) bwd_parent<2>(m, At, Xs, X, ldx, c0, cg, rg, avail, vec);
            else bwd_parent<4>(m, At, Xs, X, ldx, c0, cg, rg, avail, vec);
        } else {
            const float *xs = Xs + (size_t)off * kFuseCols;
            const int R = pick_rows(m.ns);
            if (R == 4) bwd_child<4>(m, At, xs, Xs, X, ldx, c0, cg, rg, avail, vec);
            else if (R == 2) bwd_child<2>(m, At, xs, Xs, X, ldx, c0, cg, rg, avail, vec);
            else bwd_child<1>(m, At, xs, Xs, X, ldx, c0, cg, rg, avail, vec);
            off += m.ns;
        }
        __syncthreads();  // buffer t & 1 is free
        if (t + 2 <= nk) stage_front<false>(meta[t + 2], arena, fd.relmap, nullptr, Fb + (t & 1) * max_front);
        cp_async_commit();
    }
}

template <typename T>
bool aligned16(const T *p, int ldx) {
    return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && ((size_t)ldx * sizeof(T)) % 16 == 0;
}

}  // namespace

InversePlan inverse_plan(const std::vector<int> &nf, const std::vector<int> &ns, const std::vector<int64_t> &foff) {
    InversePlan P;
    const int nodes = (int)nf.size();
    auto tiles = [](int M, int N) { return ((M + kGemmTile - 1) / kGemmTile) * ((N + kGemmTile - 1) / kGemmTile); };
    int max_ns = 0;
    for (int t = 0; t < nodes; ++t) {
        for (int b0 = 0; b0 < ns[t]; b0 += 32) P.blk.push_back(make_int2(t, b0));
        max_ns = std::max(max_ns, ns[t]);
    }
    for (int bs = 32; bs < max_ns; bs *= 2) {
        std::vector<GemmTask> p1, p2;
        int nt = 0;
        int64_t off = 0;
        for (int t = 0; t < nodes; ++t) {
            const int64_t F = foff[t];
            const int f = nf[t];
            for (int a0 = 0; a0 + bs < ns[t]; a0 += 2 * bs) {
                const int a1 = a0 + bs, a2 = std::min(a0 + 2 * bs, ns[t]), mc = a2 - a1;
                GemmTask x{};
                x.a = F + (int64_t)a0 * f + a1, x.lda = f;
                x.b = F + (int64_t)a0 * f + a0, x.ldb = f;
                x.c = off, x.ldc = mc;
                x.M = mc, x.N = bs, x.K = bs, x.flags = kGemmBUnitLower, x.tile0 = nt;
                GemmTask y{};
                y.a = F + (int64_t)a1 * f + a1, y.lda = f;
                y.b = off, y.ldb = mc;
                y.c = F + (int64_t)a0 * f + a1, y.ldc = f;
                y.M = mc, y.N = bs, y.K = mc, y.flags = kGemmAUnitLower | kGemmNeg, y.tile0 = nt;
                p1.push_back(x);
                p2.push_back(y);
                nt += tiles(mc, bs);
                off += (int64_t)mc * bs;
            }
        }
        P.scratch = std::max(P.scratch, off);
        P.p1.push_back(std::move(p1));
        P.p2.push_back(std::move(p2));
        P.tiles.push_back(nt);
    }
    int nt = 0;
    int64_t off = 0;
    for (int t = 0; t < nodes; ++t) {
        const int nb = nf[t] - ns[t];
        if (nb <= 0 || ns[t] <= 0) continue;
        const int64_t F = foff[t];
        GemmTask x{};
        x.a = F + ns[t], x.lda = nf[t];
        x.b = F, x.ldb = nf[t];
        x.c = off, x.ldc = nb;
        x.M = nb, x.N = ns[t], x.K = ns[t], x.flags = kGemmBUnitLower, x.tile0 = nt;
        GemmTask c{};
        c.a = off, c.lda = nb;
        c.c = F + ns[t], c.ldc = nf[t];
        c.M = nb, c.N = ns[t], c.tile0 = nt;
        P.w.push_back(x);
        P.wc.push_back(c);
        nt += tiles(nb, ns[t]);
        off += (int64_t)nb * ns[t];
    }
    P.wtiles = nt;
    P.scratch = std::max(P.scratch, off);
    return P;
}

template <typename T>
void inv_diag_blocks(cudaStream_t s, const FrontDev &fd, const int2 *blk, int nblk, T *arena) {
    if (nblk <= 0) return;
    k_inv_diag32<T><<<nblk, 32, 0, s>>>(fd, blk, arena);
    HSIM_LAUNCHED();
}

template <typename T>
void gemm_tasks(cudaStream_t s, const GemmTask *tasks, int ntasks, int tiles, const T *Ab, const T *Bb, T *Cb) {
    if (ntasks <= 0 || tiles <= 0) return;
    k_gemm_tasks<T><<<tiles, 256, 0, s>>>(tasks, ntasks, Ab, Bb, Cb);
    HSIM_LAUNCHED();
}

template <typename T>
void copy_tasks(cudaStream_t s, const GemmTask *tasks, int ntasks, int tiles, const T *Ab, T *Cb) {
    if (ntasks <= 0 || tiles <= 0) return;
    k_copy_tasks<T><<<tiles, 256, 0, s>>>(tasks, ntasks, Ab, Cb);
    HSIM_LAUNCHED();
}

template <typename T>
void reciprocal(cudaStream_t s, int n, const T *x, T *y) {
    if (n <= 0) return;
    k_reciprocal<T><<<cdiv(n, 256), 256, 0, s>>>(n, x, y);
    HSIM_LAUNCHED();
}

template <typename T, int STAGES>
void launch_fwd_inv(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int rt, const T *arena, int k,
                    T *X, T *Y, int ldx, bool vec) {
    constexpr size_t sm = fwd_inv_smem<T, 64>(STAGES);
    HSIM_SMEM_LIMIT_ONCE((k_solve_fwd_inv<T, 64, STAGES>), sm);
    k_solve_fwd_inv<T, 64, STAGES><<<dim3((unsigned)((int64_t)n_nodes * rt), cdiv(k, inv_cols<T>())), 256, sm, s>>>(
        fd, nodes, rt, arena, k, X, Y, ldx, vec);
    HSIM_LAUNCHED();
}

template <typename T, int BM, int STAGES>
void launch_bwd_inv(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int rt, const T *arena,
                    const T *dinv, int k, T *X, const T *Y, int ldx, bool vec, int ksplit) {
    constexpr size_t sm = bwd_inv_smem<T, BM>(STAGES);
    HSIM_SMEM_LIMIT_ONCE((k_solve_bwd_inv<T, BM, STAGES>), sm);
    if (ksplit > 1) {
        k_zero_pivot_rows<T><<<dim3((unsigned)n_nodes, 128), 256, 0, s>>>(fd, nodes, k, X, ldx);
        HSIM_LAUNCHED();
    }
    k_solve_bwd_inv<T, BM, STAGES>
        <<<dim3((unsigned)((int64_t)n_nodes * rt), cdiv(k, inv_cols<T>()), (unsigned)ksplit), 256, sm, s>>>(
            fd, nodes, rt, arena, dinv, k, X, Y, ldx, vec, ksplit);
    HSIM_LAUNCHED();
}

// SMs of the current device (queried per call: a process may drive GPUs of
// different sizes)
int device_sms() {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    return c > 0 ? c : 1;
}

// One K step per tile when every front of the height has ns <= 32 (the
// lowest heights): single-stage kernels (fewer registers, more CTAs per SM);
// otherwise the pipelined two-stage kernels.  64-row tiles also for the
// lowest heights: one 128-row tile per front (pivot rows read once) measured
// slower, 786 against 685 ms of solves per 10^6-vertex solve.
template <typename T>
void solve_fwd_inv(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int max_nf, int max_ns,
                   const T *arena, int k, T *X, T *Y, int ldx) {
    if (n_nodes <= 0 || k <= 0 || max_nf <= 0) return;
    const bool vec = aligned16(X, ldx) && aligned16(Y, ldx);
    const int rt = (max_nf + 63) / 64;
    if (max_ns <= kInvBK) launch_fwd_inv<T, 1>(s, fd, nodes, n_nodes, rt, arena, k, X, Y, ldx, vec);
    else launch_fwd_inv<T, 2>(s, fd, nodes, n_nodes, rt, arena, k, X, Y, ldx, vec);
}

template <typename T>
void solve_bwd_inv(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int max_ns, const T *arena,
                   const T *dinv, int k, T *X, const T *Y, int ldx) {
    if (n_nodes <= 0 || k <= 0 || max_ns <= 0) return;
    const bool vec = aligned16(X, ldx) && aligned16(Y, ldx);
    if (max_ns <= 32) {
        launch_bwd_inv<T, 32, 1>(s, fd, nodes, n_nodes, 1, arena, dinv, k, X, Y, ldx, vec, 1);
        return;
    }
    // heights of few large fronts fill few CTAs per SM: their long K ranges are
    // split (FP32: vector atomic additions into zeroed rows)
    const int rt = (max_ns + 63) / 64;
    const int64_t base = (int64_t)n_nodes * rt * cdiv(k, inv_cols<T>());
    int ksplit = 1;
    if (sizeof(T) == 4 && base < kBwdSplitPerSM * device_sms())
        ksplit = (int)std::min<int64_t>(kBwdMaxSplit, (kBwdSplitPerSM * device_sms() + base - 1) / base);
    launch_bwd_inv<T, 64, 2>(s, fd, nodes, n_nodes, rt, arena, dinv, k, X, Y, ldx, vec, ksplit);
}

size_t fused_smem(int max_rows, int max_front) {
    return ((size_t)max_rows * kFuseCols + 2 * (size_t)max_front) * sizeof(float);
}

int fused_max_pivots() { return kFuseMaxPiv; }
int fused_max_ancestors() { return kFuseMaxAnc; }
int fused_max_children() { return kFuseMaxKids; }
int fused_front_size(int nf, int ns) { return fuse_block(nf, ns) + pad4(nf - ns) + pad4(ns); }

FusePlan fuse_plan(const std::vector<int> &nf, const std::vector<int> &ns, const std::vector<int> &parent,
                   const std::vector<int> &h0, const std::vector<int> &h1, size_t smem_cap) {
    FusePlan F;
    F.cptr.push_back(0);
    std::vector<int> slot(nf.size(), -1);
    for (size_t i = 0; i < h1.size(); ++i) slot[h1[i]] = (int)i;
    std::vector<std::vector<int>> kids(h1.size());
    for (int t : h0)
        if (parent[t] >= 0 && slot[parent[t]] >= 0) kids[slot[parent[t]]].push_back(t);
    std::vector<char> fused(h1.size(), 0);
    for (size_t i = 0; i < h1.size(); ++i) {
        const int P = h1[i];
        int rows = nf[P], front = fused_front_size(nf[P], ns[P]);
        for (int c : kids[i]) {
            rows += ns[c];
            front = std::max(front, fused_front_size(nf[c], ns[c]));
        }
        // one launch: the largest rows and block over the fused parents size every CTA
        if (ns[P] > kFuseMaxPiv || nf[P] - ns[P] > kFuseMaxAnc || (int)kids[i].size() > kFuseMaxKids ||
            fused_smem(std::max(rows, F.rows), std::max(front, F.front)) > smem_cap) {
            F.rest1.push_back(P);
            continue;
        }
        fused[i] = 1;
        F.par.push_back(P);
        F.cid.insert(F.cid.end(), kids[i].begin(), kids[i].end());
        F.cptr.push_back((int)F.cid.size());
        F.rows = std::max(F.rows, rows);
        F.front = std::max(F.front, front);
    }
    for (int t : h0)
        if (!(parent[t] >= 0 && slot[parent[t]] >= 0 && fused[slot[parent[t]]])) F.rest0.push_back(t);
    return F;
}

void solve_fwd_fused(cudaStream_t s, const FrontDev &fd, const int *parents, int n_parents, const int *child_ptr,
                     const int *child_ids, int max_rows, int max_front, const float *arena, const float *dinv, int k,
                     float *X, float *Y, int ldx) {
    if (n_parents <= 0 || k <= 0) return;
    const size_t sm = fused_smem(max_rows, max_front);
    HSIM_SMEM_LIMIT_ONCE(k_solve_fwd_fused, kFusedSmemMax);
    HSIM_CHECK_ARG(sm <= kFusedSmemMax && max_front % 4 == 0, "fused solve: shared memory");
    const bool vec = aligned16(X, ldx) && aligned16(Y, ldx);
    k_solve_fwd_fused<<<dim3((unsigned)n_parents, cdiv(k, kFuseCols)), 256, sm, s>>>(
        fd, parents, child_ptr, child_ids, arena, dinv, k, X, Y, ldx, max_rows, max_front, vec);
    HSIM_LAUNCHED();
}

void solve_bwd_fused(cudaStream_t s, const FrontDev &fd, const int *parents, int n_parents, const int *child_ptr,
                     const int *child_ids, int max_rows, int max_front, const float *arena, int k, float *X,
                     const float *Y, int ldx) {
    if (n_parents <= 0 || k <= 0) return;
    const size_t sm = fused_smem(max_rows, max_front);
    HSIM_SMEM_LIMIT_ONCE(k_solve_bwd_fused, kFusedSmemMax);
    HSIM_CHECK_ARG(sm <= kFusedSmemMax && max_front % 4 == 0, "fused solve: shared memory");
    const bool vec = aligned16(X, ldx) && aligned16(Y, ldx);
    k_solve_bwd_fused<<<dim3((unsigned)n_parents, cdiv(k, kFuseCols)), 256, sm, s>>>(
        fd, parents, child_ptr, child_ids, arena, k, X, Y, ldx, max_rows, max_front, vec);
    HSIM_LAUNCHED();
}

#define HSIM_FINV_INSTANTIATE(T)                                                                                    \
    template void inv_diag_blocks<T>(cudaStream_t, const FrontDev &, const int2 *, int, T *);                     \
    template void gemm_tasks<T>(cudaStream_t, const GemmTask *, int, int, const T *, const T *, T *);             \
    template void copy_tasks<T>(cudaStream_t, const GemmTask *, int, int, const T *, T *);                        \
    template void reciprocal<T>(cudaStream_t, int, const T *, T *);
HSIM_FINV_INSTANTIATE(float)
HSIM_FINV_INSTANTIATE(double)
// the inverted-form solves serve the FP32 factor only
template void solve_fwd_inv<float>(cudaStream_t, const FrontDev &, const int *, int, int, int, const float *, int,
                                   float *, float *, int);
template void solve_bwd_inv<float>(cudaStream_t, const FrontDev &, const int *, int, int, const float *,
                                   const float *, int, float *, const float *, int);

}  // namespace k
}  // namespace hsim
