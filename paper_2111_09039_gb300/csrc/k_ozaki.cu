// FP64-accurate dense products on BF16 tensor cores (error-free splitting).
//
// The Gram products S_bar = Psi^T S Psi, M_bar = Psi^T M Psi and the basis
// update Phi = Psi Phi_bar of Alg. 1 are the dominant dense work of the
// subspace iteration; in FP64 they run at the GB300's 1.2 TFLOP/s FP64 rate.
// Here each FP64 operand is split, against one power of two per row (or per
// column), into kSlices integer digits of at most 8 bits,
//     x = 2^(e-7) * sum_s d_s 2^(-8 s),   |d_0| <= 128, |d_s| <= 128,
// which BF16 represents exactly.  A digit product is an integer of at most
// 2^14, so up to 1024 of them sum exactly in an FP32 accumulator: the tensor
// cores compute sum_r d_s(x_ir) d_t(y_jr) with no rounding, grouped by
// D = s + t (pairs with D >= kSlices are dropped), over K-chunks of 128, and
// every chunk is flushed into FP64 registers.  The result equals the FP64
// product up to the dropped tail, about 2^-47 of max|x_i.| max|y_j.| per
// term.
//
// Kernel shape: C (FP64, M x N) (+)= X Y^T with X (M x K) and Y (N x K) both
// K-contiguous digit slices; CTA tile 64 x 64, eight warps of 16 x 32,
// mma.sync m16n8k16 BF16 with FP32 accumulation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "common.h"
#include "kernels.h"

namespace hsim {
namespace k {

namespace {

constexpr int kSlices = kOzakiSlices;
constexpr int TM = 64, TN = 64, TKs = 32;   // CTA tile and K step
constexpr int kPad = 8;                      // smem row padding (bf16)
constexpr int kRow = TKs + kPad;             // 40 bf16 = 80 bytes per smem row
constexpr int kFlush = 128;                  // K rows between FP32 -> FP64 flushes

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// exponent e with max|x| < 2^e (frexp convention); -1074 for all-zero groups
__device__ __forceinline__ int exp_of(double a) {
    if (a == 0.0) return -1074;
    int e;
    frexp(a, &e);
    return e;
}

// per-row exponents of a row-major R x C FP64 block: one warp per row
__global__ void k_row_exps(int R, int C, const double *__restrict__ X, int ldx, int *__restrict__ ex) {
    int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (row >= R) return;
    double m = 0.0;
    for (int j = lane; j < C; j += 32) m = fmax(m, fabs(X[(size_t)row * ldx + j]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) ex[row] = exp_of(m);
}

// per-column exponents of a row-major R x C FP64 block (ex pre-set to -1074)
__global__ void k_col_exps(int R, int C, const double *__restrict__ X, int ldx, int *__restrict__ ex) {
    const int r0 = blockIdx.x * 256;
    const int r1 = min(R, r0 + 256);
    for (int j = blockIdx.y * blockDim.x + threadIdx.x; j < C; j += gridDim.y * blockDim.x) {
        double m = 0.0;
        for (int r = r0; r < r1; ++r) m = fmax(m, fabs(X[(size_t)r * ldx + j]));
        if (m != 0.0) atomicMax(&ex[j], exp_of(m));
    }
}

__device__ __forceinline__ void split_value(double x, int e, __nv_bfloat16 *out, size_t stride) {
    // y = x 2^-e in (-1, 1); digits d_0 = rint(128 y), then 256 * remainder
    double y = ldexp(x, 7 - e);
    double d = rint(y);
    out[0] = __double2bfloat16(d);
    double r = y - d;
#pragma unroll
    for (int s = 1; s < kSlices; ++s) {
        r *= 256.0;
        d = rint(r);
        out[(size_t)s * stride] = __double2bfloat16(d);
        r -= d;
    }
}

// slices of a row-major R x C block split per row: out[s] is R x ldo (K = C
// contiguous), columns C..ldo-1 zero
__global__ void k_split_rows(int R, int C, const double *__restrict__ X, int ldx, const int *__restrict__ ex,
                             __nv_bfloat16 *__restrict__ out, int ldo, size_t slice_stride) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)R * ldo) return;
    int i = (int)(idx / ldo), j = (int)(idx % ldo);
    double x = j < C ? X[(size_t)i * ldx + j] : 0.0;
    split_value(x, ex[i], out + (size_t)i * ldo + j, slice_stride);
}

// slices of a row-major R x C block split per column, transposed: out[s] is
// C x ldo with K = R contiguous (rows R..ldo-1 zero)
__global__ void k_split_cols_t(int R, int C, const double *__restrict__ X, int ldx, const int *__restrict__ ex,
                               __nv_bfloat16 *__restrict__ out, int ldo, size_t slice_stride) {
    __shared__ double tile[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int r = r0 + yy, c = c0 + threadIdx.x;
        tile[yy][threadIdx.x] = (r < R && c < C) ? X[(size_t)r * ldx + c] : 0.0;
    }
    __syncthreads();
    for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
        int c = c0 + yy, r = r0 + threadIdx.x;
        if (c < C && r < ldo) split_value(tile[threadIdx.x][yy], ex[c], out + (size_t)c * ldo + r, slice_stride);
    }
}

__global__ void k_fill_int(int n, int v, int *__restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3, unsigned addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(smem)), "l"(gmem),
                 "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;\n" ::); }

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

constexpr int kStageElems = kSlices * (TM + TN) * kRow;  // bf16 per pipeline stage

// C[i0.., j0..] (+)= 2^(ex_i + ey_j - 14) sum_D 2^(-8 D) sum_{s+t=D} X_s Y_t^T over
// rows k in [k_beg, k_end).  X slices: M x ldx, Y slices: N x ldy (K contiguous,
// ld multiples of 8, zero padded to a multiple of TKs).  Two pipeline stages
// filled with cp.async; each 128-row chunk of exact FP32 digit sums is added
// into an FP32 (hi, lo) pair per output with TwoSum.
__global__ void __launch_bounds__(256, 1)
    k_ozaki_nt(int M, int N, const __nv_bfloat16 *__restrict__ Xs, int ldx, size_t xstride,
               const __nv_bfloat16 *__restrict__ Ys, int ldy, size_t ystride, const int *__restrict__ ex,
               const int *__restrict__ ey, double *__restrict__ C, int ldc, int k_len, int k_split, int atomic,
               int lower) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16 *stage0 = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
    const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;
    // lower: only tiles that meet the lower triangle j <= i (square tiles)
    if (lower && j0 > i0 + TM - 1) return;
    const int k_beg = blockIdx.z * k_split;
    const int k_end = min(k_len, k_beg + k_split);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp & 3, wn = warp >> 2;  // warp tile rows wm*16, cols wn*32
    float acc[kSlices][4][4];
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int d = 0; d < kSlices; ++d)
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[d][t][e] = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) hi[t][e] = lo[t][e] = 0.f;

    // stage the K step starting at kk into buffer `buf`: every slice of the
    // 64 x 32 X and Y blocks, 16-byte chunks, zero-filled outside the operands
    auto load_stage = [&](int buf, int kk) {
        __nv_bfloat16 *As = stage0 + (size_t)buf * kStageElems;
        __nv_bfloat16 *Bs = As + (size_t)kSlices * TM * kRow;
        constexpr int chunks = kSlices * TM * (TKs / 8);  // per operand
        for (int c = threadIdx.x; c < 2 * chunks; c += blockDim.x) {
            const bool isB = c >= chunks;
            const int cc = isB ? c - chunks : c;
            const int s = cc / (TM * (TKs / 8));
            const int rem = cc % (TM * (TKs / 8));
            const int row = rem / (TKs / 8), part = rem % (TKs / 8);
            const int grow = (isB ? j0 : i0) + row;
            const int lim = isB ? N : M;
            const bool ok = grow < lim && kk + part * 8 < k_end;
            const __nv_bfloat16 *src = isB ? Ys + (size_t)s * ystride + (size_t)(ok ? grow : 0) * ldy + (ok ? kk + part * 8 : 0)
                                           : Xs + (size_t)s * xstride + (size_t)(ok ? grow : 0) * ldx + (ok ? kk + part * 8 : 0);
            __nv_bfloat16 *dst = (isB ? Bs : As) + ((size_t)s * TM + row) * kRow + part * 8;
            cp_async16(dst, src, ok ? 16 : 0);
        }
    };

    int buf = 0;
    if (k_beg < k_end) load_stage(0, k_beg);
    cp_async_commit();
    int since_flush = 0;
    for (int kk = k_beg; kk < k_end; kk += TKs) {
        if (kk + TKs < k_end) load_stage(buf ^ 1, kk + TKs);
        cp_async_commit();
        cp_async_wait_1();
        __syncthreads();
        const __nv_bfloat16 *As = stage0 + (size_t)buf * kStageElems;
        const __nv_bfloat16 *Bs = As + (size_t)kSlices * TM * kRow;
#pragma unroll
        for (int k16 = 0; k16 < TKs; k16 += 16) {
            unsigned a[kSlices][4];
#pragma unroll
            for (int s = 0; s < kSlices; ++s) {
                const int r = wm * 16 + (lane & 15);
                const int c = k16 + (lane >> 4) * 8;
                ldsm_x4(a[s][0], a[s][1], a[s][2], a[s][3], smem_addr(As + ((size_t)s * TM + r) * kRow + c));
            }
#pragma unroll
            for (int t = 0; t < kSlices; ++t) {
                unsigned b[4][2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    // n rows wn*32 + h*16 + (0..15), k halves by lane groups
                    const int nrow = wn * 32 + h * 16 + ((lane >> 4) << 3) + (lane & 7);
                    const int c = k16 + ((lane >> 3) & 1) * 8;
                    ldsm_x4(b[2 * h][0], b[2 * h][1], b[2 * h + 1][0], b[2 * h + 1][1],
                            smem_addr(Bs + ((size_t)t * TN + nrow) * kRow + c));
                }
#pragma unroll
                for (int s = 0; s + t < kSlices; ++s)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[s + t][nt], a[s], b[nt][0], b[nt][1]);
            }
        }
        __syncthreads();
        buf ^= 1;
        since_flush += TKs;
        if (since_flush >= kFlush || kk + TKs >= k_end) {
            since_flush = 0;
#pragma unroll
            for (int d = 0; d < kSlices; ++d) {
                const float w = __int_as_float((127 - 8 * d) << 23);  // 2^(-8 d), exact
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        two_sum_acc(hi[t][e], lo[t][e], __fmul_rn(acc[d][t][e], w));
                        acc[d][t][e] = 0.f;
                    }
            }
        }
    }
    cp_async_wait_0();
    // epilogue: C fragment (row g / g+8, cols 2*tig + {0,1}) per n-tile
    const int g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = i0 + wm * 16 + g + (e >= 2 ? 8 : 0);
            const int j = j0 + wn * 32 + nt * 8 + tig * 2 + (e & 1);
            if (i < M && j < N && (!lower || j <= i)) {
                const double v = ldexp((double)hi[nt][e] + (double)lo[nt][e], ex[i] + ey[j] - 14);
                if (atomic) atomicAdd(&C[(size_t)i * ldc + j], v);
                else C[(size_t)i * ldc + j] = v;
                if (lower && j < i) {
                    if (atomic) atomicAdd(&C[(size_t)j * ldc + i], v);
                    else C[(size_t)j * ldc + i] = v;
                }
            }
        }
}

size_t smem_bytes() { return 2 * (size_t)kStageElems * sizeof(__nv_bfloat16); }

int sm_count_oz() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

void launch_nt(cudaStream_t s, int M, int N, const __nv_bfloat16 *Xs, int ldx, size_t xstride,
               const __nv_bfloat16 *Ys, int ldy, size_t ystride, const int *ex, const int *ey, double *C, int ldc,
               int k_len, int splits, int lower) {
    // the kernel reads the digit slices as 16-byte vectors: every slice base
    // and every row start must be 16-byte aligned
    auto aligned16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    HSIM_CHECK_ARG(aligned16(Xs) && aligned16(Ys) && ldx % 8 == 0 && ldy % 8 == 0 && xstride % 8 == 0 &&
                       ystride % 8 == 0 && k_len % TKs == 0,
                   "ozaki product: operand not 16-byte aligned");
    HSIM_CHECK_ARG(!lower || (M == N && TM == TN), "ozaki product: lower triangle needs a square result");
    const size_t sm = smem_bytes();
    HSIM_CUDA(cudaFuncSetAttribute(k_ozaki_nt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int k_split = (int)((k_len + splits - 1) / splits);
    k_split = (k_split + kFlush - 1) / kFlush * kFlush;
    splits = (int)cdiv(k_len, k_split);
    dim3 g(cdiv(N, TN), cdiv(M, TM), (unsigned)splits);
    k_ozaki_nt<<<g, 256, sm, s>>>(M, N, Xs, ldx, xstride, Ys, ldy, ystride, ex, ey, C, ldc, k_len, k_split,
                                  splits > 1 ? 1 : 0, lower);
    HSIM_LAUNCHED();
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

}  // namespace

// Scratch sizes are whole multiples of 256 bytes, so operands placed back to
// back in one buffer keep the 16-byte alignment of the vector loads.
size_t ozaki_cols_scratch(int n, int cols) {
    const int ldk = round_up(n, TKs);
    size_t b = (size_t)kSlices * cols * ldk * sizeof(__nv_bfloat16) + sizeof(int) * (size_t)cols;
    return (b + 511) / 256 * 256;
}

size_t ozaki_rows_scratch(int rows, int k) {
    const int ldk = round_up(k, TKs);
    size_t b = (size_t)kSlices * rows * ldk * sizeof(__nv_bfloat16) + sizeof(int) * (size_t)rows;
    return (b + 511) / 256 * 256;
}

OzakiOperand ozaki_split_cols(cudaStream_t s, int n, int cols, const double *X, int ldx, void *scratch) {
    OzakiOperand op;
    op.rows = cols;
    op.ld = round_up(n, TKs);
    op.stride = (size_t)cols * op.ld;
    op.slices = static_cast<__nv_bfloat16 *>(scratch);
    op.exps = reinterpret_cast<int *>(op.slices + (size_t)kSlices * op.stride);
    if (n <= 0 || cols <= 0) return op;
    k_fill_int<<<cdiv(cols, 256), 256, 0, s>>>(cols, -1074, op.exps);
    HSIM_LAUNCHED();
    k_col_exps<<<dim3(cdiv(n, 256), cdiv(cols, 256)), 256, 0, s>>>(n, cols, X, ldx, op.exps);
    HSIM_LAUNCHED();
    k_split_cols_t<<<dim3(cdiv(op.ld, 32), cdiv(cols, 32)), dim3(32, 8), 0, s>>>(n, cols, X, ldx, op.exps,
                                                                                  op.slices, op.ld, op.stride);
    HSIM_LAUNCHED();
    return op;
}

OzakiOperand ozaki_split_rows(cudaStream_t s, int rows, int k, const double *X, int ldx, void *scratch) {
    OzakiOperand op;
    op.rows = rows;
    op.ld = round_up(k, TKs);
    op.stride = (size_t)rows * op.ld;
    op.slices = static_cast<__nv_bfloat16 *>(scratch);
    op.exps = reinterpret_cast<int *>(op.slices + (size_t)kSlices * op.stride);
    if (rows <= 0) return op;
    k_row_exps<<<cdiv(rows, 8), 256, 0, s>>>(rows, k, X, ldx, op.exps);
    HSIM_LAUNCHED();
    k_split_rows<<<cdiv((int64_t)rows * op.ld, 256), 256, 0, s>>>(rows, k, X, ldx, op.exps, op.slices, op.ld,
                                                                  op.stride);
    HSIM_LAUNCHED();
    return op;
}

void ozaki_product(cudaStream_t s, const OzakiOperand &X, const OzakiOperand &Y, int k_len, double *C, int ldc,
                   int splits, bool lower) {
    if (X.rows <= 0 || Y.rows <= 0) return;
    HSIM_CHECK_ARG(X.ld == Y.ld, "ozaki_product: operands split over different K");
    if (splits <= 0) {
        const int64_t tx = cdiv(X.rows, TM), ty = cdiv(Y.rows, TN);
        const int64_t tiles = lower ? tx * (tx + 1) / 2 : tx * ty;
        splits = (int)std::max<int64_t>(1, std::min<int64_t>((4LL * sm_count_oz() + tiles - 1) / tiles,
                                                              (int64_t)cdiv(k_len, 1024)));
    }
    if (splits > 1) {
        if (ldc == Y.rows) HSIM_CUDA(cudaMemsetAsync(C, 0, (size_t)X.rows * Y.rows * sizeof(double), s));
        else HSIM_CUDA(cudaMemset2DAsync(C, (size_t)ldc * sizeof(double), 0, (size_t)Y.rows * sizeof(double), X.rows, s));
    }
    launch_nt(s, X.rows, Y.rows, X.slices, X.ld, X.stride, Y.slices, Y.ld, Y.stride, X.exps, Y.exps, C, ldc, X.ld,
              splits, lower ? 1 : 0);
}

}  // namespace k
}  // namespace hsim
