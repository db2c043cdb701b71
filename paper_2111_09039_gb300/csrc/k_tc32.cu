// FP32-accurate dense tile products on the tcgen05 tensor cores (kind::tf32),
// for the mixed path's FP32 factorisation and many-right-hand-side solves
// (Sec. 3.2, direct solver; Alg. 1 factors K = S - mu M once per level and
// solves with it in every inverse iteration).
//
// Every product here is C (+)= A B over an output tile of BM x BN = 128 x 128
// FP32 values, K staged BK = 32 at a time through two shared-memory stages:
// all 256 threads load the next stage's FP32 operands from global memory
// (the layouts of fronts and right-hand-side rows are irregular, so no bulk
// copies), split each value into two TF32 halves, x = hi + lo (hi the
// nearest TF32 value, lo the nearest TF32 value to the FP32 remainder), and
// store them in the K-major core-matrix order the tensor cores read, while
// one thread issues the MMAs of the current stage:
//     D += A_hi B_hi + A_hi B_lo + A_lo B_hi        (3 MMAs per 8-deep K step)
// with D a 128-lane x 128-column FP32 accumulator in TMEM.  The dropped
// A_lo B_lo and the rounding of lo leave about 2^-21 of sum |a b| (an FP32
// product leaves about 2^-24 per term); the inverse iterations run in
// correction form, so this error is relative to the residual.  After the
// last stage the accumulator is read back (tcgen05.ld) by all eight warps
// and the epilogue of the operation stores, subtracts or scatters it.
//
// Shared-memory layout of one operand half (R = 128 rows x BK = 32 K, FP32
// bit patterns): K-major with the 128-byte swizzle, one 128-byte row per
// operand row (its 32 K values), 8-row atoms of 1024 bytes, the 16-byte chunk
// q (K values 4q .. 4q + 3) of row r at chunk q ^ (r % 8):
//     byte offset(r, k) = (r / 8) * 1024 + (r % 8) * 128 + ((k / 4) ^ (r % 8)) * 16 + (k % 4) * 4.
// Each 8-deep MMA step starts 32 bytes further into the rows.  A thread writes
// one row's 4 consecutive K values as one 16-byte store; with the swizzle,
// the 8 threads of a quarter warp hit 8 different chunk columns whether they
// hold 8 rows of one K quad or 8 K quads of one row, so each operand is
// loaded with the thread mapping that makes its global reads coalesce: lanes
// along the rows for operands whose rows are contiguous in memory (columns of
// a front, right-hand-side rows), lanes along K for operands whose K index is
// contiguous (B(kk, j) = B[j ldb + kk] of the inversion products).
//
// Operations (functors below): the forward products of the inverted-form
// solves (k_finv.cu) for the tree heights with the largest fronts, the
// batched products of the pivot-block inversion (GemmTask lists), and the
// rank-128 Schur-complement updates of the blocked factorisation of large
// fronts.  The same engine measured slower than the CUDA-core kernels for the
// backward products (K over all rows of few large fronts) and for rank-32
// updates (one K step per tile), which therefore stay on the CUDA cores.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "common.h"
#include "kernels.h"
#include "tc.h"

namespace hsim {
namespace k {

namespace {

constexpr int BM = 128, BN = 128, BK = 32, THREADS = 256;
constexpr uint32_t HALF_BYTES = BM * BK * 4;       // 16 KB: one operand half of one stage
constexpr uint32_t STAGE_BYTES = 4 * HALF_BYTES;   // A_hi, A_lo, B_hi, B_lo
constexpr size_t SMEM = 2 * (size_t)STAGE_BYTES + 1024;
constexpr uint32_t TMEM_COLS = BN;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s per barrier wait

__device__ int g_tc32_error;

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

__device__ __forceinline__ uint32_t swz_off(int r, int kq) {
    return (uint32_t)(r >> 3) * 1024u + (uint32_t)(r & 7) * 128u + (uint32_t)((kq ^ r) & 7) * 16u;
}

// (row, K quad) of this thread's item it (0..3) of a 128 x 32 operand: lanes
// along rows (row-contiguous operands) or along the 8 K quads
template <bool KCONTIG>
__device__ __forceinline__ void item(int tid, int it, int &m, int &kq) {
    const int idx = tid + THREADS * it;
    if (KCONTIG) {
        kq = idx & 7;
        m = idx >> 3;
    } else {
        m = idx & (BM - 1);
        kq = idx >> 7;
    }
}

__device__ __forceinline__ void sts_v4(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// 32 consecutive outputs of one row, plain or accumulated atomically with a sign
__device__ __forceinline__ void store32(float *p, const float (&v)[32], int avail, bool vec) {
    if (vec && avail >= 32) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            reinterpret_cast<float4 *>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int c = 0; c < 32; ++c)
            if (c < avail) p[c] = v[c];
    }
}
__device__ __forceinline__ void atomic_sub32(float *p, const float (&v)[32], int avail, bool vec) {
    if (vec && avail >= 32) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            atomicAdd(reinterpret_cast<float4 *>(p) + q,
                      make_float4(-v[4 * q], -v[4 * q + 1], -v[4 * q + 2], -v[4 * q + 3]));
    } else {
#pragma unroll
        for (int c = 0; c < 32; ++c)
            if (c < avail) atomicAdd(p + c, -v[c]);
    }
}

// ---- the tile engine ----------------------------------------------------------

template <class Op>
__global__ void __launch_bounds__(THREADS, 1) k_tc32(const Op op) {
    extern __shared__ unsigned char smem_dyn[];
    __shared__ __align__(8) uint64_t bar[2], done;
    __shared__ uint32_t tmem_slot;
    typename Op::Tile T;
    if (!op.tile(T)) return;  // depends on blockIdx only: uniform over the CTA
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nk = T.ke > T.kb ? (T.ke - T.kb + BK - 1) / BK : 0;
    const uint32_t smem0 = (tc::smem_addr(smem_dyn) + 1023u) & ~1023u;
    int *err = &g_tc32_error;
    if (tid == 0) {
        tc::mbar_init(tc::smem_addr(&bar[0]), 1);
        tc::mbar_init(tc::smem_addr(&bar[1]), 1);
        tc::mbar_init(tc::smem_addr(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         tc::smem_addr(&tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // this thread's 4 (row, K quad) items of A and of B per stage
    float ra[4][4], rb[4][4];
    auto load = [&](int k0) {
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            int m, kq;
            item<Op::kAKContig>(tid, it, m, kq);
#pragma unroll
            for (int q = 0; q < 4; ++q) ra[it][q] = op.a(T, m, k0 + 4 * kq + q);
            item<Op::kBKContig>(tid, it, m, kq);
#pragma unroll
            for (int q = 0; q < 4; ++q) rb[it][q] = op.b(T, m, k0 + 4 * kq + q);
        }
    };
    auto store = [&](int st) {
        const uint32_t base = smem0 + (uint32_t)st * STAGE_BYTES;
#pragma unroll
        for (int it = 0; it < 4; ++it) {
            int m, kq;
            float h[4], l[4];
            item<Op::kAKContig>(tid, it, m, kq);
            uint32_t off = swz_off(m, kq);
#pragma unroll
            for (int q = 0; q < 4; ++q) tc::tf32_split(ra[it][q], h[q], l[q]);
            sts_v4(base + off, h[0], h[1], h[2], h[3]);
            sts_v4(base + HALF_BYTES + off, l[0], l[1], l[2], l[3]);
            item<Op::kBKContig>(tid, it, m, kq);
            off = swz_off(m, kq);
#pragma unroll
            for (int q = 0; q < 4; ++q) tc::tf32_split(rb[it][q], h[q], l[q]);
            sts_v4(base + 2 * HALF_BYTES + off, h[0], h[1], h[2], h[3]);
            sts_v4(base + 3 * HALF_BYTES + off, l[0], l[1], l[2], l[3]);
        }
    };
    constexpr uint32_t idesc = tc::idesc_tf32(BM, BN);
    bool ok = true;
    if (nk > 0) {
        load(T.kb);
        store(0);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
        const int st = kt & 1;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t base = smem0 + (uint32_t)st * STAGE_BYTES;
#pragma unroll
            for (int k8 = 0; k8 < BK / 8; ++k8) {
                const uint32_t o = (uint32_t)k8 * 32;  // 8 TF32 values further along the rows
                const uint64_t ah = tc::smem_desc_sw128(base + o);
                const uint64_t al = tc::smem_desc_sw128(base + HALF_BYTES + o);
                const uint64_t bh = tc::smem_desc_sw128(base + 2 * HALF_BYTES + o);
                const uint64_t bl = tc::smem_desc_sw128(base + 3 * HALF_BYTES + o);
                tc::mma_tf32(tmem, al, bh, idesc, (kt > 0 || k8 > 0) ? 1 : 0);
                tc::mma_tf32(tmem, ah, bl, idesc, 1);
                tc::mma_tf32(tmem, ah, bh, idesc, 1);
            }
            tc::commit(tc::smem_addr(&bar[st]));
        }
        if (kt + 1 < nk) {
            load(T.kb + (kt + 1) * BK);
            // stage st ^ 1 was last read by the MMAs of step kt - 1
            if (kt >= 1 && ok) ok = tc::mbar_wait(tc::smem_addr(&bar[st ^ 1]), ((kt - 1) >> 1) & 1, err, WAIT_NS);
            store(st ^ 1);
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        }
        __syncthreads();
    }
    if (nk > 0) {
        // every MMA has completed before TMEM is read or freed (also after a
        // timed-out wait above)
        if (tid == 0) tc::commit(tc::smem_addr(&done));
        ok = tc::mbar_wait(tc::smem_addr(&done), 0, err, WAIT_NS) && ok;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile rows), columns
    // 64 (w / 4) .. + 63 in two 32-column loads
    const int quad = warp & 3, c_half = warp >> 2;
    const int m = 32 * quad + lane;
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
        const int n0 = 64 * c_half + 32 * j;
        float v[32];
        if (nk > 0) {
            uint32_t r[32];
            tc::tmem_ld32(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)n0, r);
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
        } else {
#pragma unroll
            for (int c = 0; c < 32; ++c) v[c] = 0.f;
        }
        if (ok) op.store(T, m, n0, v);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

// ---- operations ---------------------------------------------------------------

// Forward product of one tree height (CTA = front x 128-row tile x 128
// columns): out(r, c) = sum_{j < ns} A(r, j) X(ps + j, c), A = Linv (unit
// lower) on the pivot rows and W below; rows r < ns go to Y, rows r >= ns are
// subtracted from the ancestors' rows of X (siblings share them).
struct FwdSolveOp {
    static constexpr bool kAKContig = false, kBKContig = false;  // front columns, X rows
    FrontDev fd;
    const int *nodes;
    int rt, k, ldx;
    const float *arena;
    float *X, *Y;
    bool vec;
    struct Tile {
        int nf, ns, ps, r0, c0, kb, ke;
        const float *F;
        const int *rows;
    };
    __device__ bool tile(Tile &T) const {
        const int t = nodes[blockIdx.x / rt];
        T.r0 = (int)(blockIdx.x % rt) * BM;
        T.nf = fd.nf[t];
        T.ns = fd.ns[t];
        if (T.r0 >= T.nf || T.ns == 0) return false;
        T.ps = fd.pstart[t];
        T.c0 = blockIdx.y * BN;
        T.F = arena + fd.foff[t];
        T.rows = fd.rows + fd.rows_off[t];
        T.kb = 0;
        T.ke = (T.r0 + BM <= T.ns) ? T.r0 + BM : T.ns;  // Linv(r, j) = 0 for j > r
        return true;
    }
    __device__ float a(const Tile &T, int m, int j) const {
        const int r = T.r0 + m;
        if (r >= T.nf || j >= T.ke) return 0.f;
        if (r >= T.ns || r > j) return T.F[(int64_t)j * T.nf + r];
        return r == j ? 1.f : 0.f;
    }
    __device__ float b(const Tile &T, int n, int j) const {
        const int c = T.c0 + n;
        if (j >= T.ke || c >= k) return 0.f;
        return X[(int64_t)(T.ps + j) * ldx + c];
    }
    __device__ void store(const Tile &T, int m, int n0, const float (&v)[32]) const {
        const int r = T.r0 + m, c = T.c0 + n0, avail = k - c;
        if (r >= T.nf || avail <= 0) return;
        if (r < T.ns) store32(Y + (int64_t)(T.ps + r) * ldx + c, v, avail, vec);
        else atomic_sub32(X + (int64_t)T.rows[r] * ldx + c, v, avail, vec);
    }
};

// Batched products of the pivot-block inversion: C = sg A B for every task
// (A, B, C column-major at the task's offsets; unit-lower operands implied),
// the tasks' tiles numbered consecutively in 128 x 128 tiles (tile0).
__device__ __forceinline__ int find_task_tc(const GemmTask *tasks, int ntasks, int tile) {
    int lo = 0, hi = ntasks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].tile0 <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct GemmTaskOp {
    static constexpr bool kAKContig = false, kBKContig = true;  // A(i, kk) = A[kk lda + i], B(kk, j) = B[j ldb + kk]
    const GemmTask *tasks;
    int ntasks;
    const float *Ab, *Bb;
    float *Cb;
    struct Tile {
        GemmTask tk;
        int m0, n0, kb, ke;
    };
    __device__ bool tile(Tile &T) const {
        T.tk = tasks[find_task_tc(tasks, ntasks, blockIdx.x)];
        const int local = blockIdx.x - T.tk.tile0;
        const int ntn = (T.tk.N + BN - 1) / BN;
        T.m0 = (local / ntn) * BM;
        T.n0 = (local % ntn) * BN;
        // a unit lower A has A(i, kk) = 0 for kk > i; a unit lower B has B(kk, j) = 0 for kk < j
        T.kb = (T.tk.flags & kGemmBUnitLower) ? T.n0 : 0;
        T.ke = (T.tk.flags & kGemmAUnitLower) ? min(T.tk.K, T.m0 + BM) : T.tk.K;
        return true;
    }
    __device__ float a(const Tile &T, int m, int kk) const {
        const int i = T.m0 + m;
        if (i >= T.tk.M || kk >= T.ke) return 0.f;
        if (T.tk.flags & kGemmAUnitLower) return i > kk ? Ab[T.tk.a + (int64_t)kk * T.tk.lda + i] : (i == kk ? 1.f : 0.f);
        return Ab[T.tk.a + (int64_t)kk * T.tk.lda + i];
    }
    __device__ float b(const Tile &T, int n, int kk) const {
        const int j = T.n0 + n;
        if (j >= T.tk.N || kk >= T.ke) return 0.f;
        if (T.tk.flags & kGemmBUnitLower) return kk > j ? Bb[T.tk.b + (int64_t)j * T.tk.ldb + kk] : (kk == j ? 1.f : 0.f);
        return Bb[T.tk.b + (int64_t)j * T.tk.ldb + kk];
    }
    __device__ void store(const Tile &T, int m, int n0, const float (&v)[32]) const {
        const int i = T.m0 + m;
        if (i >= T.tk.M) return;
        const float sg = (T.tk.flags & kGemmNeg) ? -1.f : 1.f;
        float *C = Cb + T.tk.c + i;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const int j = T.n0 + n0 + c;
            if (j < T.tk.N) C[(int64_t)j * T.tk.ldc] = sg * v[c];
        }
    }
};

// Schur-complement update after a block of kSchurBlock pivot columns [K0, K0
// + kSchurBlock) of the blocked FP32 factorisation (CTA = one 128 x 128 tile
// (m0, n0) of a front's trailing part, which starts at column K0 +
// kSchurBlock): F(r, c) -= sum_kk L(r, K0 + kk) d_kk L(c, K0 + kk) for r >= c,
// d_kk the pivot on the diagonal, L the unit-lower factor's columns below it.
struct SchurOp {
    static constexpr bool kAKContig = false, kBKContig = false;  // front columns (rows contiguous)
    FrontDev fd;
    const SchurTask *tasks;
    int K0;
    float *arena;
    struct Tile {
        float *F;
        int nf, r0, c0, kb, ke;
    };
    __device__ bool tile(Tile &T) const {
        const SchurTask tk = tasks[blockIdx.x];
        T.nf = fd.nf[tk.node];
        T.F = arena + fd.foff[tk.node];
        T.r0 = K0 + kSchurBlock + tk.m0;
        T.c0 = K0 + kSchurBlock + tk.n0;
        T.kb = 0;
        T.ke = min(kSchurBlock, fd.ns[tk.node] - K0);
        return T.ke > 0 && T.r0 < T.nf && T.c0 < T.nf;
    }
    __device__ float a(const Tile &T, int m, int kk) const {
        const int r = T.r0 + m;
        if (r >= T.nf || kk >= T.ke) return 0.f;
        return T.F[(int64_t)(K0 + kk) * T.nf + r];
    }
    __device__ float b(const Tile &T, int n, int kk) const {
        const int c = T.c0 + n;
        if (c >= T.nf || kk >= T.ke) return 0.f;
        const float *col = T.F + (int64_t)(K0 + kk) * T.nf;
        return col[c] * col[K0 + kk];
    }
    __device__ void store(const Tile &T, int m, int n0, const float (&v)[32]) const {
        const int r = T.r0 + m;
        if (r >= T.nf) return;
#pragma unroll
        for (int cc = 0; cc < 32; ++cc) {
            const int c = T.c0 + n0 + cc;
            if (c < T.nf && r >= c) T.F[(int64_t)c * T.nf + r] -= v[cc];
        }
    }
};

template <class Op>
void launch(cudaStream_t s, dim3 grid, const Op &op) {
    HSIM_SMEM_LIMIT_ONCE(k_tc32<Op>, SMEM);
    k_tc32<Op><<<grid, THREADS, SMEM, s>>>(op);
    HSIM_LAUNCHED();
}

bool aligned16f(const float *p, int ldx) {
    return (reinterpret_cast<uintptr_t>(p) % 16 == 0) && ((size_t)ldx * sizeof(float)) % 16 == 0;
}

}  // namespace

void solve_fwd_tc(cudaStream_t s, const FrontDev &fd, const int *nodes, int n_nodes, int max_nf, const float *arena,
                  int k, float *X, float *Y, int ldx) {
    if (n_nodes <= 0 || k <= 0 || max_nf <= 0) return;
    FwdSolveOp op{fd, nodes, (int)cdiv(max_nf, BM), k, ldx, arena, X, Y, aligned16f(X, ldx) && aligned16f(Y, ldx)};
    launch(s, dim3((unsigned)((int64_t)n_nodes * op.rt), cdiv(k, BN)), op);
}

void schur_tc(cudaStream_t s, const FrontDev &fd, const SchurTask *tasks, int ntasks, int K0, float *arena) {
    if (ntasks <= 0) return;
    launch(s, dim3((unsigned)ntasks), SchurOp{fd, tasks, K0, arena});
}

void gemm_tasks_tc(cudaStream_t s, const GemmTask *tasks, int ntasks, int tiles, const float *Ab, const float *Bb,
                   float *Cb) {
    if (ntasks <= 0 || tiles <= 0) return;
    launch(s, dim3((unsigned)tiles), GemmTaskOp{tasks, ntasks, Ab, Bb, Cb});
}

int gemm_tiles_tc(std::vector<GemmTask> &tasks) {
    int nt = 0;
    for (auto &t : tasks) {
        t.tile0 = nt;
        nt += (int)(cdiv(t.M, BM) * cdiv(t.N, BN));
    }
    return nt;
}

void tc32_check(cudaStream_t s) {
    int h = 0;
    HSIM_CUDA(cudaMemcpyFromSymbolAsync(&h, g_tc32_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaStreamSynchronize(s));
    if (h != 0) {
        const int zero = 0;
        HSIM_CUDA(cudaMemcpyToSymbolAsync(g_tc32_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
        HSIM_CUDA(cudaStreamSynchronize(s));
        fail(HSIM_E_TIMEOUT, "tensor-core FP32 product: an mbarrier wait timed out");
    }
}

}  // namespace k
}  // namespace hsim
