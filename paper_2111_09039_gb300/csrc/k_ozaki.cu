// FP64-accurate dense products on BF16 tensor cores (error-free splitting).
//
// The Gram products S_bar = Psi^T S Psi, M_bar = Psi^T M Psi and the basis
// update Phi = Psi Phi_bar of Alg. 1 are the dominant dense work of the
// subspace iteration; in FP64 they run at the GB300's 1.2 TFLOP/s FP64 rate.
// Here each FP64 operand is split, against one power of two per row (or per
// column), into SL integer digits of at most 8 bits (SL = 6, or 5 where 39
// bits suffice),
//     x = 2^(e-7) * sum_s d_s 2^(-8 s),   |d_0| <= 128, |d_s| <= 128,
// which BF16 represents exactly.  A digit product is an integer of at most
// 2^14, so up to 1024 of them sum exactly in an FP32 accumulator: the tensor
// cores compute sum_r d_s(x_ir) d_t(y_jr) with no rounding, grouped by
// D = s + t (pairs with D >= SL are dropped).  The sum for D = SL - 1 takes
// SL digit pairs per K row, so K-chunks of flush_k<SL>() rows (192 for five
// digits, 160 for six: at most 1024 / SL, a multiple of the 32-row stage)
// stay exact, and every chunk is flushed into FP32 TwoSum pairs.  The result equals the FP64
// product up to the dropped tail, about 2^-(8 SL - 1) of max|x_i.| max|y_j.|
// per term (2^-47 with six digits).
//
// Kernel shape: C (FP64, M x N) (+)= X Y^T with X (M x K) and Y (N x K) both
// K-contiguous digit slices, on the tcgen05 tensor cores (TMA-fed shared
// memory, TMEM accumulators; k_ozaki_tc below).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.h"
#include "fpconv.h"
#include "kernels.h"

namespace hsim {
namespace k {

namespace {

constexpr int kSlices = kOzakiSlices;  // the most digits an operand holds (scratch sizing)
constexpr int TKs = 32;      // K padding of the digit slices (one pipeline stage)

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Exponents and digits are taken from the bits of the FP64 values with integer
// arithmetic only (the FP64 pipe of this part is ~1/60 of the FP32 pipe).
//
// exponent e with |x| < 2^e for a nonzero x: biased exponent - 1022 (exact
// for normal numbers, an upper bound for subnormals); -1074 marks zero
__device__ __forceinline__ int exp_bits(double a) {
    const long long b = __double_as_longlong(a) & 0x7FFFFFFFFFFFFFFFLL;
    if (b == 0) return -1074;
    return (int)(b >> 52) - 1022;
}

// per-row exponents of a row-major R x C FP64 block: one warp per row
__global__ void k_row_exps(int R, int C, const double *__restrict__ X, int ldx, int *__restrict__ ex) {
    int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (row >= R) return;
    int m = -1074;
    for (int j = lane; j < C; j += 32) m = max(m, exp_bits(X[(size_t)row * ldx + j]));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) ex[row] = m;
}

// per-column exponents of a row-major R x C FP64 block (ex pre-set to -1074)
__global__ void k_col_exps(int R, int C, const double *__restrict__ X, int ldx, int *__restrict__ ex) {
    const int r0 = blockIdx.x * 256;
    const int r1 = min(R, r0 + 256);
    for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < C; j += gridDim.y * blockDim.x) {
        int m = -1074;
        for (int r = r0; r < r1; ++r) m = max(m, exp_bits(X[(size_t)r * ldx + j]));
        if (m != -1074) atomicMax(&ex[j], m);
    }
}

// Digits of x against the group exponent e (|x| < 2^e): T = round(x 2^(B-e)),
// B = 8 SL - 1, as an integer (|T| <= 2^B, ties to even), written in balanced
// base 256,
//     T = sum_s d_s 2^(8 (SL - 1 - s)),  d_1..d_{SL-1} in [-128, 127],  |d_0| <= 128,
// so x = 2^(e-7) sum_s d_s 2^(-8 s) up to 2^(e-B-1).
template <int SL>
__device__ __forceinline__ void split_value(double x, int e, __nv_bfloat16 *out, size_t stride) {
    const long long bits = __double_as_longlong(x);
    int E = (int)((bits >> 52) & 0x7FF);
    long long M = bits & 0xFFFFFFFFFFFFFLL;
    if (E == 0) E = 1;
    else M |= 1LL << 52;
    const int sh = E - 1075 + (8 * SL - 1) - e;  // x 2^(B-e) = +-M 2^sh, sh <= B - 53 when |x| < 2^e
    long long T = 0;
    if (M != 0 && sh > -54) {
        if (sh >= 0) {
            T = M << min(sh, 10);
        } else {
            const int k = -sh;
            long long q = M >> k;
            const long long rem = M & ((1LL << k) - 1), half = 1LL << (k - 1);
            if (rem > half || (rem == half && (q & 1))) ++q;
            T = q;
        }
    }
    if (bits < 0) T = -T;
#pragma unroll
    for (int s = SL - 1; s >= 1; --s) {
        int d = (int)(T & 255);
        if (d >= 128) d -= 256;
        out[(size_t)s * stride] = __int2bfloat16_rn(d);
        T = (T - d) >> 8;
    }
    out[0] = __int2bfloat16_rn((int)T);
}

// Global layout of the digit slices ("tiled"): for K-chunk kc = k / 32,
// slice s, row r (rows padded to rows_p, a multiple of 128) and k,
//     offset = ((kc * SL + s) * rows_p + 8 (r / 8)) * 32 + 64 ((k % 32) / 8)
//              + 8 (r % 8) + k % 8     (BF16 elements),
// i.e. 8 x 8 core matrices (8 rows x 16 bytes) ordered [kc][s][r/8][k%32/8].
// A 32-deep K step of any 128 (or 64) consecutive rows of one slice is then
// one contiguous 8 KB (4 KB) block that a bulk copy moves straight into the
// core-matrix order the tensor-core descriptors read.
template <int SL>
__device__ __forceinline__ size_t tiled_off(int s, int r, int k, int rows_p) {
    return (((size_t)(k >> 5) * SL + s) * (size_t)rows_p + (size_t)(r & ~7)) * 32 + (size_t)((k & 31) >> 3) * 64 +
           (size_t)(r & 7) * 8 + (size_t)(k & 7);
}

// digits of the 8 values v[0..7] (consecutive k of one row, exponent e) as
// one 16-byte vector per slice
template <int SL>
__device__ __forceinline__ void split8_store(const double (&v)[8], int e, __nv_bfloat16 *out, size_t off,
                                             int rows_p) {
    __nv_bfloat16 d[SL][8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        __nv_bfloat16 one[SL];
        split_value<SL>(v[t], e, one, 1);
#pragma unroll
        for (int sl = 0; sl < SL; ++sl) d[sl][t] = one[sl];
    }
    const size_t slice_step = (size_t)rows_p * 32;  // next slice within the same K-chunk
#pragma unroll
    for (int sl = 0; sl < SL; ++sl)
        *reinterpret_cast<uint4 *>(out + off + sl * slice_step) = *reinterpret_cast<const uint4 *>(d[sl]);
}

// split a row-major R x K block per row (K = columns): one thread per row and
// 8-wide K group; a warp covers one 8-row group x one 32-deep K-chunk
template <int SL>
__global__ void k_split_rows_tiled(int R, int K, const double *__restrict__ X, int ldx, const int *__restrict__ ex,
                                   __nv_bfloat16 *__restrict__ out, int rows_p, int kp) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int KC = kp / 32;
    if (gw >= (int64_t)(rows_p / 8) * KC) return;
    const int rg = (int)(gw / KC), kc = (int)(gw % KC);
    const int r = rg * 8 + (lane & 7), k0 = kc * 32 + (lane >> 3) * 8;
    double v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = (r < R && k0 + t < K) ? X[(size_t)r * ldx + k0 + t] : 0.0;
    split8_store<SL>(v, r < R ? ex[r] : -1074, out, tiled_off<SL>(0, r, k0, rows_p), rows_p);
}

// split a row-major K x C block per column (operand row r = column r, K =
// rows of X), transposed through shared memory: a block handles 32 columns x
// a 32-deep K-chunk
template <int SL>
__global__ void k_split_cols_tiled(int K, int C, const double *__restrict__ X, int ldx, const int *__restrict__ ex,
                                   __nv_bfloat16 *__restrict__ out, int rows_p) {
    __shared__ double tile[32][33];
    const int kc = blockIdx.x, c0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 4 threads
    for (int yy = ty; yy < 32; yy += 4) {
        const int k = kc * 32 + yy, c = c0 + tx;
        tile[yy][tx] = (k < K && c < C) ? X[(size_t)k * ldx + c] : 0.0;
    }
    __syncthreads();
    // thread -> (column c0 + lc, K group kg): 32 columns x 4 groups = 128 threads
    const int lc = (threadIdx.x & 7) + 8 * (threadIdx.x >> 5), kg = (threadIdx.x >> 3) & 3;
    const int r = c0 + lc;
    if (r >= rows_p) return;
    double v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = tile[kg * 8 + t][lc];
    split8_store<SL>(v, r < C ? ex[r] : -1074, out, tiled_off<SL>(0, r, kc * 32 + kg * 8, rows_p), rows_p);
}

__global__ void k_fill_int(int n, int v, int *__restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// Error-free accumulation of x into (hi, lo): hi + lo gains x exactly up to
// the rounding of lo (Knuth's TwoSum in FP32; the FP32 pipe is ~60x the FP64
// pipe on this part).
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x) {
    float s = __fadd_rn(hi, x);
    float bp = __fsub_rn(s, hi);
    float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// SMs of the current device (queried per call: a process may drive GPUs of
// different sizes; the attribute query costs about a microsecond)
int sm_count_oz() {
    int dev = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    return c > 0 ? c : 1;
}

// tcgen05 form of the same product (5th-generation tensor cores, TMEM).
//
// CTA tile: 128 rows of X by 64 rows of Y, K staged 32 at a time into three
// shared-memory stages by bulk copies (TMA, cp.async.bulk): the tiled global
// layout makes each slice of a stage one contiguous block, so a stage is 6
// copies of 8 KB (X) and 6 of 4 KB (Y), landing in core-matrix order
// [s][r/8][k/8][8 x 16 bytes]: an MMA operand descriptor with LBO = 128 bytes
// between K-groups and SBO = 512 bytes between 8-row groups.  Because the Y
// slices of one stage follow each other at the row-group stride, Y_0 .. Y_5
// form one N = 384 operand: one MMA multiplies X_s by [Y_0 .. Y_{5-s}] (N = 64 (6 - s),
// split at 256) and its 64-column blocks land exactly on the accumulators
// acc_{s} .. acc_{5} of the digit sums D = s + t, which sit side by side in
// TMEM (columns 64 D .. 64 D + 63, 384 of the 512 allocated).  Per 16-deep
// K step that is 8 MMAs instead of 21.
//
// Warp roles (320 threads): warp 0 issues the TMA loads, warp 1 owns the
// TMEM allocation and issues the MMAs (one thread), warps 2..9 drain TMEM:
// after every exact-FP32 chunk of flush_k<SL>() K rows they read acc_0..acc_5 and
// add 2^-8D acc_D into FP32 (hi, lo) TwoSum pairs held in registers, one
// TMEM lane (output row) and 32 of the 64 columns per thread.  Every wait on an mbarrier gives up
// after a bounded number of polls, records an error flag the host checks,
// and the CTA still drains its own copies and MMAs and frees its TMEM.
// ---------------------------------------------------------------------------
constexpr int TC_M = 128, TC_N = 64, TC_K = 32, TC_STAGES = 3;
constexpr int TC_THREADS = 320, TC_DRAIN = 256;  // 10 warps, 8 of them drain TMEM
constexpr int TC_KG = TC_K / 8;
// K rows per exact FP32 chunk: SL digit pairs per row for the sum D = SL - 1,
// each at most 2^14, so chunk x SL <= 1024 keeps the FP32 sums exact
template <int SL> __host__ __device__ constexpr int flush_k() { return (1024 / SL) / TC_K * TC_K; }
static_assert(flush_k<5>() == 192 && flush_k<6>() == 160, "exact chunk lengths");
// stage sizes for SL digit slices: X 128 rows, Y 64 rows (SL = 6: 49,152 + 24,576 bytes)
template <int SL> __host__ __device__ constexpr uint32_t tc_a_bytes() { return 16u * TC_M * SL * TC_KG; }
template <int SL> __host__ __device__ constexpr uint32_t tc_b_bytes() { return 16u * TC_N * SL * TC_KG; }
template <int SL> __host__ __device__ constexpr uint32_t tc_stage_bytes() { return tc_a_bytes<SL>() + tc_b_bytes<SL>(); }
template <int SL> constexpr size_t tc_smem() { return (size_t)TC_STAGES * tc_stage_bytes<SL>() + 1024; }
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr uint64_t TC_WAIT_NS = 2000000000ull;  // 2 s per barrier wait

__device__ int g_oz_error;

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    // shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29),
    // SBO >> 4 (32-45), descriptor version 1 (bits 46-47), no swizzle (61-63 = 0)
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t umma_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// wait for the phase of the given parity; gives up after TC_WAIT_NS of wall time
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if ((it & 255u) == 0) {
            const uint64_t t = global_ns();
            if (it == 0) t0 = t;
            else if (t - t0 > TC_WAIT_NS) break;
        }
    }
    atomicExch(&g_oz_error, 1);
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// bulk copy (TMA) of `bytes` contiguous bytes global -> shared, completing on bar
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void umma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
        "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

template <int SL>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_ozaki_tc(int M, int N, const __nv_bfloat16 *__restrict__ Xs, int rows_px, const __nv_bfloat16 *__restrict__ Ys,
               int rows_py, const int *__restrict__ ex, const int *__restrict__ ey, double *__restrict__ C, int ldc,
               int k_len, int k_split, int atomic, int lower) {
    extern __shared__ unsigned char smem_dyn[];
    __shared__ __align__(8) uint64_t full_bar[TC_STAGES], empty_bar[TC_STAGES], accf_bar, acce_bar, drain_bar;
    __shared__ uint32_t tmem_slot;
    const int i0 = blockIdx.y * TC_M, j0 = blockIdx.x * TC_N;
    if (lower && j0 > i0 + TC_M - 1) return;
    const int k_beg = blockIdx.z * k_split;
    const int k_end = min(k_len, k_beg + k_split);
    const int nk = k_end > k_beg ? (k_end - k_beg) / TC_K : 0;
    constexpr int kFlush = flush_k<SL>();
    const int nchunks = (nk + (kFlush / TC_K) - 1) / (kFlush / TC_K);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // stages on a 1024-byte boundary
    const uint32_t smem0 = (smem_addr(smem_dyn) + 1023u) & ~1023u;
    if (threadIdx.x == 0) {
        for (int st = 0; st < TC_STAGES; ++st) {
            mbar_init(smem_addr(&full_bar[st]), 1);
            mbar_init(smem_addr(&empty_bar[st]), 1);
        }
        mbar_init(smem_addr(&accf_bar), 1);
        mbar_init(smem_addr(&acce_bar), TC_DRAIN);
        mbar_init(smem_addr(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_slot)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0 && nk > 0) {
            // producer: stage kt % 3 is refilled once the MMAs of kt - 3 completed
            bool ok = true;
            int issued = 0;
            for (int kt = 0; kt < nk && ok; ++kt) {
                const int st = kt % TC_STAGES;
                if (kt >= TC_STAGES) ok = mbar_wait(smem_addr(&empty_bar[st]), ((kt / TC_STAGES) & 1) ^ 1);
                if (!ok) break;
                const uint32_t fb = smem_addr(&full_bar[st]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(tc_stage_bytes<SL>())
                             : "memory");
                const uint32_t a_dst = smem0 + st * tc_stage_bytes<SL>();
                const size_t kc = (size_t)(k_beg + kt * TC_K) / TC_K;
#pragma unroll 1
                for (int sl = 0; sl < SL; ++sl) {
                    bulk_load(a_dst + sl * (tc_a_bytes<SL>() / SL),
                              Xs + ((kc * SL + sl) * rows_px + i0) * TC_K, tc_a_bytes<SL>() / SL, fb);
                    bulk_load(a_dst + tc_a_bytes<SL>() + sl * (tc_b_bytes<SL>() / SL),
                              Ys + ((kc * SL + sl) * rows_py + j0) * TC_K, tc_b_bytes<SL>() / SL, fb);
                }
                issued = kt + 1;
            }
            // drain: the last loads of every stage have landed before the CTA exits
            for (int kt = max(0, issued - TC_STAGES); kt < issued; ++kt)
                mbar_wait(smem_addr(&full_bar[kt % TC_STAGES]), (kt / TC_STAGES) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0 && nk > 0) {
            bool ok = true;
            // core matrices: 128 bytes apart along K, 512 bytes apart along rows
            constexpr uint32_t LBO = 128, SBO = 512;
            for (int kt = 0; kt < nk && ok; ++kt) {
                const int st = kt % TC_STAGES;
                const int chunk = kt / (kFlush / TC_K);
                const bool chunk_first = kt % (kFlush / TC_K) == 0;
                ok = mbar_wait(smem_addr(&full_bar[st]), (kt / TC_STAGES) & 1);
                if (ok && chunk_first && chunk > 0) ok = mbar_wait(smem_addr(&acce_bar), (chunk - 1) & 1);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t a_base = smem0 + st * tc_stage_bytes<SL>(), b_base = a_base + tc_a_bytes<SL>();
#pragma unroll
                for (int k16 = 0; k16 < TC_K / 16; ++k16) {
                    const uint32_t a_k = a_base + 2 * k16 * LBO, b_k = b_base + 2 * k16 * LBO;
#pragma unroll
                    for (int sl = 0; sl < SL; ++sl) {
                        const uint64_t ad = umma_desc(a_k + sl * (tc_a_bytes<SL>() / SL), LBO, SBO);
                        const int acc = (chunk_first && k16 == 0 && sl == 0) ? 0 : 1;
                        const int ncols = TC_N * (SL - sl);  // Y_0 .. Y_{SL-1-s}
                        const int n1 = ncols > 256 ? 256 : ncols;
                        umma_f16(tmem + TC_N * sl, ad, umma_desc(b_k, LBO, SBO), umma_idesc(TC_M, n1), acc);
                        if (ncols > 256)  // rows 256.. of [Y_0 .. Y_5]: 32 row groups further
                            umma_f16(tmem + TC_N * sl + 256, ad, umma_desc(b_k + 32u * SBO, LBO, SBO),
                                     umma_idesc(TC_M, ncols - 256), acc);
                    }
                }
                umma_commit(smem_addr(&empty_bar[st]));
                if (kt % (kFlush / TC_K) == (kFlush / TC_K) - 1 || kt == nk - 1) umma_commit(smem_addr(&accf_bar));
            }
            // every MMA issued by this thread has completed before teardown
            umma_commit(smem_addr(&drain_bar));
            mbar_wait(smem_addr(&drain_bar), 0);
        }
    } else {
        // drain warps: TMEM lane quadrant = warp % 4, one output row and one
        // 32-column half per thread
        const int quad = warp & 3, c0 = 32 * ((warp - 2) >> 2);
        const int row = 32 * quad + lane;
        float hi[32], lo[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) hi[c] = lo[c] = 0.f;
        bool ok = true;
        for (int ch = 0; ch < nchunks && ok; ++ch) {
            ok = mbar_wait(smem_addr(&accf_bar), ch & 1);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int d = 0; d < SL; ++d) {
                const float w = __int_as_float((127 - 8 * d) << 23);  // 2^(-8 d), exact
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(32 * quad) << 16) + TC_N * d + c0, r);
#pragma unroll
                for (int c = 0; c < 32; ++c) two_sum_acc(hi[c], lo[c], __fmul_rn(__uint_as_float(r[c]), w));
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(smem_addr(&acce_bar));
        }
        const int i = i0 + row;
        if (ok && i < M) {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const int j = j0 + c0 + c;
                if (j < N && (!lower || j <= i)) {
                    // exact conversions and the power-of-two scaling on the
                    // bit patterns: one FP64 instruction per output
                    const double v = scale2(f2d_bits(hi[c]) + f2d_bits(lo[c]), ex[i] + ey[j] - 14);
                    if (atomic) atomicAdd(&C[(size_t)i * ldc + j], v);
                    else C[(size_t)i * ldc + j] = v;
                    if (lower && j < i) {
                        if (atomic) atomicAdd(&C[(size_t)j * ldc + i], v);
                        else C[(size_t)j * ldc + i] = v;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS));
}

template <int SL>
void launch_tc(cudaStream_t s, int M, int N, const __nv_bfloat16 *Xs, int rows_px, const __nv_bfloat16 *Ys,
               int rows_py, const int *ex, const int *ey, double *C, int ldc, int k_len, int splits, int lower) {
    auto aligned16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    HSIM_CHECK_ARG(aligned16(Xs) && aligned16(Ys) && rows_px % TC_M == 0 && rows_py % TC_M == 0 && M <= rows_px &&
                       N <= rows_py && k_len % TC_K == 0,
                   "ozaki product: operand layout not supported");
    HSIM_CHECK_ARG(!lower || M == N, "ozaki product: lower triangle needs a square result");
    HSIM_SMEM_LIMIT_ONCE(k_ozaki_tc<SL>, tc_smem<SL>());
    int k_split = (int)((k_len + splits - 1) / splits);
    constexpr int kFlush = flush_k<SL>();
    k_split = (k_split + kFlush - 1) / kFlush * kFlush;
    splits = (int)cdiv(k_len, k_split);
    dim3 g(cdiv(N, TC_N), cdiv(M, TC_M), (unsigned)splits);
    k_ozaki_tc<SL><<<g, TC_THREADS, tc_smem<SL>(), s>>>(M, N, Xs, rows_px, Ys, rows_py, ex, ey, C, ldc, k_len, k_split,
                                               splits > 1 ? 1 : 0, lower);
    HSIM_LAUNCHED();
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

// Scratch: (up to) kSlices x rows_p x kp BF16 digits (tiled layout) then rows_p
// exponents, rounded to whole 256-byte blocks so operands placed back to back
// in one buffer stay aligned for the bulk copies.
static size_t operand_bytes(int rows, int kdim) {
    const size_t rows_p = (size_t)round_up(std::max(rows, 1), TC_M), kp = (size_t)round_up(std::max(kdim, 1), TKs);
    size_t b = (size_t)kSlices * rows_p * kp * sizeof(__nv_bfloat16) + sizeof(int) * rows_p;
    return (b + 511) / 256 * 256;
}

size_t ozaki_cols_scratch(int n, int cols) { return operand_bytes(cols, n); }
size_t ozaki_rows_scratch(int rows, int k) { return operand_bytes(rows, k); }

static OzakiOperand make_operand(int rows, int kdim, void *scratch, int digits) {
    HSIM_CHECK_ARG(digits == 5 || digits == 6, "ozaki product: 5 or 6 digits per value");
    OzakiOperand op;
    op.digits = digits;
    op.rows = rows;
    op.rows_p = round_up(std::max(rows, 1), TC_M);
    op.kp = round_up(std::max(kdim, 1), TKs);
    op.slices = static_cast<__nv_bfloat16 *>(scratch);
    op.exps = reinterpret_cast<int *>(op.slices + (size_t)digits * op.rows_p * op.kp);
    return op;
}

OzakiOperand ozaki_split_cols(cudaStream_t s, int n, int cols, const double *X, int ldx, void *scratch, int digits) {
    OzakiOperand op = make_operand(cols, n, scratch, digits);
    if (n <= 0 || cols <= 0) return op;
    k_fill_int<<<cdiv(cols, 256), 256, 0, s>>>(cols, -1074, op.exps);
    HSIM_LAUNCHED();
    k_col_exps<<<dim3(cdiv(n, 256), cdiv(cols, 256)), 256, 0, s>>>(n, cols, X, ldx, op.exps);
    HSIM_LAUNCHED();
    const dim3 g(op.kp / 32, cdiv(op.rows_p, 32));
    if (digits == 5) k_split_cols_tiled<5><<<g, 128, 0, s>>>(n, cols, X, ldx, op.exps, op.slices, op.rows_p);
    else k_split_cols_tiled<6><<<g, 128, 0, s>>>(n, cols, X, ldx, op.exps, op.slices, op.rows_p);
    HSIM_LAUNCHED();
    return op;
}

OzakiOperand ozaki_split_rows(cudaStream_t s, int rows, int k, const double *X, int ldx, void *scratch, int digits) {
    OzakiOperand op = make_operand(rows, k, scratch, digits);
    if (rows <= 0) return op;
    k_row_exps<<<cdiv(rows, 8), 256, 0, s>>>(rows, k, X, ldx, op.exps);
    HSIM_LAUNCHED();
    const int64_t warps = (int64_t)(op.rows_p / 8) * (op.kp / 32);
    if (digits == 5)
        k_split_rows_tiled<5><<<cdiv(warps * 32, 256), 256, 0, s>>>(rows, k, X, ldx, op.exps, op.slices, op.rows_p,
                                                                   op.kp);
    else
        k_split_rows_tiled<6><<<cdiv(warps * 32, 256), 256, 0, s>>>(rows, k, X, ldx, op.exps, op.slices, op.rows_p,
                                                                   op.kp);
    HSIM_LAUNCHED();
    return op;
}

void ozaki_product(cudaStream_t s, const OzakiOperand &X, const OzakiOperand &Y, int k_len, double *C, int ldc,
                   int splits, bool lower) {
    if (X.rows <= 0 || Y.rows <= 0) return;
    HSIM_CHECK_ARG(X.kp == Y.kp, "ozaki_product: operands split over different K");
    HSIM_CHECK_ARG(X.digits == Y.digits, "ozaki_product: operands split into different digit counts");
    if (splits <= 0) {
        // split K so that tiles x splits fills whole waves of one CTA per SM
        const int64_t tx = cdiv(X.rows, TC_M), ty = cdiv(Y.rows, TC_N);
        int64_t tiles = 0;
        for (int64_t r = 0; r < tx; ++r) tiles += lower ? std::min<int64_t>(ty, (r * TC_M + TC_M - 1) / TC_N + 1) : ty;
        const int64_t sms = sm_count_oz();
        const int64_t s_max = std::max<int64_t>(1, std::min<int64_t>(k_len / 2048, 8 * sms / tiles + 1));
        double best = -1.0;
        splits = 1;
        for (int64_t sp = 1; sp <= s_max; ++sp) {
            const int64_t ctas = tiles * sp, waves = (ctas + sms - 1) / sms;
            // fill of the last wave, with a small preference for fewer splits
            const double eff = (double)ctas / (double)(waves * sms) - 0.002 * (double)sp;
            if (sp * tiles >= sms / 2 && eff > best + 1e-9) {
                best = eff;
                splits = (int)sp;
            }
        }
        if (best < 0) splits = (int)s_max;
    }
    if (splits > 1) {
        if (ldc == Y.rows) HSIM_CUDA(cudaMemsetAsync(C, 0, (size_t)X.rows * Y.rows * sizeof(double), s));
        else HSIM_CUDA(cudaMemset2DAsync(C, (size_t)ldc * sizeof(double), 0, (size_t)Y.rows * sizeof(double), X.rows, s));
    }
    if (X.digits == 5)
        launch_tc<5>(s, X.rows, Y.rows, X.slices, X.rows_p, Y.slices, Y.rows_p, X.exps, Y.exps, C, ldc, X.kp, splits,
                     lower ? 1 : 0);
    else
        launch_tc<6>(s, X.rows, Y.rows, X.slices, X.rows_p, Y.slices, Y.rows_p, X.exps, Y.exps, C, ldc, X.kp, splits,
                     lower ? 1 : 0);
}

void ozaki_check(cudaStream_t s) {
    int h = 0;
    HSIM_CUDA(cudaMemcpyFromSymbolAsync(&h, g_oz_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaStreamSynchronize(s));
    if (h != 0) {
        const int zero = 0;
        HSIM_CUDA(cudaMemcpyToSymbolAsync(g_oz_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s));
        HSIM_CUDA(cudaStreamSynchronize(s));
        fail(HSIM_E_INTERNAL, "tensor-core product: an mbarrier wait timed out");
    }
}

}  // namespace k
}  // namespace hsim
