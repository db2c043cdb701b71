// HSIM driver and C ABI.
//
// hsim_build_hierarchy: host construction of the vertex hierarchy, the
//   prolongations and every level's symbolic analysis (Sec. 4.1, Alg. 2).
// hsim_solve: the hot path, all on the GPU (Alg. 3):
//   Galerkin products S^tau, M^tau -> dense coarsest eigenproblem ->
//   for tau = T-2 .. 0: prolongation U Phi, shift mu = Lambda_floor(alpha p),
//   numeric LDL^T of S - mu M, subspace iterations (Alg. 1: two inverse
//   iterations, Rayleigh-Ritz with FP64 Jacobi, update, convergence test of
//   eq. conv2, locking) until the p lowest pairs have converged.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <functional>
#include <future>
#include <initializer_list>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <type_traits>
#include <utility>
#include <vector>

#include "common.h"
#include "host.h"
#include "kernels.h"

namespace hsim {
std::atomic<uint64_t> g_launches{0};
}

using namespace hsim;

namespace {
thread_local std::string g_last_error;

// HSIM_TRACE=1 prints one line per subspace iteration to stderr.
int trace_level() {
    static const int lv = [] {
        const char *e = std::getenv("HSIM_TRACE");
        return (e && *e) ? std::atoi(e) : 0;
    }();
    return lv;
}
bool trace_on() { return trace_level() > 0; }

hsim_status guard(const std::function<void()> &f) {
    try {
        f();
        return HSIM_OK;
    } catch (const Error &e) {
        g_last_error = e.what();
        return e.status;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return HSIM_E_NOMEM;
    } catch (const std::exception &e) {
        g_last_error = e.what();
        return HSIM_E_INTERNAL;
    }
}
}  // namespace

void hsim::set_last_error(const std::string &msg) { g_last_error = msg; }

namespace {
// Kernels read the caller's arrays through raw pointers: plain host memory
// or memory of another device is refused here, before any launch.  Pinned
// or managed memory is accepted (the device reaches it); a pointer the
// runtime cannot classify is let through unchanged.
void check_device_ptrs(int device, std::initializer_list<std::pair<const char *, const void *>> ptrs) {
    for (const auto &np : ptrs) {
        if (!np.second) continue;
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, np.second) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        HSIM_CHECK_ARG(a.type != cudaMemoryTypeUnregistered,
                       std::string(np.first) + " is host memory; a device pointer is expected");
        HSIM_CHECK_ARG(a.type != cudaMemoryTypeDevice || a.device == device,
                       std::string(np.first) + " lives on device " + std::to_string(a.device) +
                           ", not on the context's device " + std::to_string(device));
    }
}
}  // namespace

struct hsim_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    DevBuf<int> flags;        // small device flag area
    std::vector<int> hflags;  // host mirror
    DevBuf<unsigned long long> scratch_u64;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) HSIM_CUDA(cudaSetDevice(dev));
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

struct LevelData {
    int n = 0;
    bool dense = false;
    Csr pat_nat;                 // natural-order pattern
    std::vector<int64_t> vmap;   // internal entry -> natural entry
    Csr pat_int;                 // internal-order pattern
    DevCsr dpat;                 // internal pattern on the device
    DevBuf<int64_t> dvmap;
    DevBuf<int> drow_of;         // row of each internal entry
    FrontSymbolic fs;
    DevBuf<int64_t> d_foff, d_rows_off, d_relmap_off, d_asm;
    DevBuf<int> d_nf, d_ns, d_pstart, d_rows, d_relmap, d_parent, d_perm, d_iperm, d_hnodes, d_ea;
    std::vector<int64_t> hnodes_off, ea_off;
    std::vector<std::vector<int>> step_cnt, step_maxnf;
    std::vector<int> ea_maxu;
    k::FrontDev fd{};
    // inverted-factor solves: largest nf and ns per tree height; the
    // inversion's 32 x 32 diagonal blocks, its block-doubling levels (two
    // products each) and the product W = L_bs Linv with its copy-back
    std::vector<int> h_maxnf, h_maxns;
    DevBuf<int2> inv_blk;
    int n_inv_blk = 0;
    std::vector<DevBuf<k::GemmTask>> inv_p1, inv_p2;
    std::vector<int> inv_n, inv_tiles;
    DevBuf<k::GemmTask> inv_w, inv_wc;
    int inv_nw = 0, inv_tw = 0;
    // the same tasks numbered in 128 x 128 tiles for the tensor-core products
    // (FP32 factors): block-doubling levels, and the W products of fronts with
    // at least kTcMinPivots pivots (the others stay on the CUDA cores)
    std::vector<DevBuf<k::GemmTask>> inv_p1_tc, inv_p2_tc;
    std::vector<int> inv_tiles_tc;
    DevBuf<k::GemmTask> inv_w_tc, inv_w_cc;
    int inv_nw_tc = 0, inv_tw_tc = 0, inv_nw_cc = 0, inv_tw_cc = 0;
    int64_t inv_scratch = 0;
    // blocked FP32 factorisation of the heights with fronts of kTcMinSchurFront
    // or more: per height and block of kSchurBlock pivot columns, the offset of
    // its trailing-update tiles in schur_tasks (schur_off[h].size() = blocks + 1;
    // empty: the height is factored panel by panel)
    std::vector<std::vector<int64_t>> schur_off;
    DevBuf<k::SchurTask> schur_tasks;
    // FP32 solves of heights 0 and 1 in one launch each way: the fused fronts
    // of height 1 with their children (fuse_cid[fuse_cptr[i] ..
    // fuse_cptr[i + 1])), the leaves and height-1 fronts solved per height
    DevBuf<int> fuse_par, fuse_cptr, fuse_cid, fuse_rest0, fuse_rest1;
    int fuse_n = 0, fuse_n0 = 0, fuse_n1 = 0, fuse_rows = 0, fuse_front = 0;
};

struct ProlongData {
    Csr U_nat;    // rows: level tau natural, cols: level tau+1 natural
    Csr U_int;    // internal orders
    Csr Ut_int;   // transpose (with values)
    Csr T_pat;    // pattern of S_int^tau U_int
    DevCsr dU, dUt, dT;
    DevBuf<double> dUval, dUtval;
    double rho = 0.0;
    int fallback = 0;
};

}  // namespace

struct hsim_hier {
    hsim_ctx *ctx = nullptr;
    int device = 0;
    int n = 0, m = 0, p = 0, T = 0;  // n: level-0 unknowns
    int n_mesh = 0;                    // mesh vertices (n unless a Dirichlet boundary removes some)
    hsim_options opts{};
    std::vector<int> sizes, order;
    std::vector<int> dofs;             // Dirichlet: mesh id of each level-0 unknown (empty: identity)
    std::vector<LevelData> lev;
    std::vector<ProlongData> pro;
    // level-0 pattern of S (natural order) and the assembly data; with a
    // Dirichlet boundary the assembly runs on the whole mesh's pattern patm,
    // then S and M are gathered into pat0 (maps d_smap, d_dofs)
    DevCsr pat0, patm;
    DevBuf<int64_t> d_smap;
    DevBuf<int> d_dofs;
    DevBuf<int> dF, d_ecot, d_vt_ptr, d_vt_idx, d_diag_ptr, d_diag_col;
    // workspaces, grown on demand
    DevBuf<double> S0int, M0int, Md0int, dinv0, arena, dpos, ritz_work, Sbar, Mbar, lam, phibar, res_sums,
        Phi, Psi, SP, MP, coarseX, coarseLam, colw, tmpv, signs, tval_s, tval_m;
    std::vector<DevBuf<double>> Sv, Mv;  // level values (internal), index tau
    // mixed precision: FP32 factor and FP32 right-hand-side blocks
    DevBuf<float> arena32, dpos32, X32;
    // inverted-factor solves: 1 / D, the forward result Y, inversion scratch
    DevBuf<double> dinvf, ysol, invs;
    DevBuf<float> dinvf32, ysol32, invs32;
    DevBuf<double> rho;
    DevBuf<unsigned char> oz;  // digit slices of the tensor-core products
};

namespace {

// Device copies of the front inversion's tasks (k::inverse_plan) and the
// per-height maxima of nf and ns for the inverted-factor solves.
// Tensor-core FP32 products (k_tc32.cu) replace the CUDA-core kernels of the
// FP32 factorisation and solves where they measured faster (10^6-vertex
// level 0, 750 right-hand sides): the block-doubling inversion levels of 64
// and more and the W products of fronts with at least kTcMinPivots pivots
// (factor and inversion 1.1 ms faster), and the forward products of tree
// heights whose fronts reach kTcMinFwdPivots pivots (0.6 ms faster per
// solve).  The backward products (K runs over all nf rows of few large
// fronts) and the rank-32 Schur updates of the right-looking factorisation
// (one 32-deep K step per tile) measured slower on the tensor cores (+2.6 and
// +8 ms) and stay on the CUDA cores.  HSIM_TC32=0 keeps every FP32 product on
// the CUDA cores (for comparison; read at every factorisation and solve).
constexpr int kTcMinPivots = 128, kTcMinFwdPivots = 300;
// FP32 factorisation: heights whose largest front has this many rows are
// factored in blocks of k::kSchurBlock pivot columns, the trailing update of
// each block on the tensor cores (rank kSchurBlock instead of rank 32)
constexpr int kTcMinSchurFront = 512;
// mixed path: the Grams take 5 digits per value at tolerances from this up, 6 below
constexpr double kGramFiveDigitTol = 1e-6;
bool tc32_enabled() {
    const char *e = std::getenv("HSIM_TC32");
    return !(e && *e == '0');
}
// FP32 solves: each front of height 1 with its leaves in one CTA per column
// tile (k::solve_fwd_fused / solve_bwd_fused), for parents whose CTA needs at
// most k::kFuseSmemCap bytes of shared memory (three CTAs per SM); the others
// per height.  HSIM_FUSE=0 solves every height separately (for comparison;
// read at every solve).
bool fuse_enabled() {
    const char *e = std::getenv("HSIM_FUSE");
    return !(e && *e == '0');
}

int number_tiles(std::vector<k::GemmTask> &tasks, int tile) {
    int nt = 0;
    for (auto &t : tasks) {
        t.tile0 = nt;
        nt += ((t.M + tile - 1) / tile) * ((t.N + tile - 1) / tile);
    }
    return nt;
}

// Heights 0 and 1 of the FP32 solves: the fronts of height 1 of k::fuse_plan
// solved with their children (all leaves) in one CTA, the rest per height.
// Not planned when either height reaches the tensor-core forward products.
void build_fuse_plan(LevelData &L, cudaStream_t s) {
    const FrontSymbolic &fs = L.fs;
    L.fuse_n = L.fuse_n0 = L.fuse_n1 = L.fuse_rows = L.fuse_front = 0;
    if (fs.max_height < 1 || L.h_maxns[0] >= kTcMinFwdPivots || L.h_maxns[1] >= kTcMinFwdPivots) return;
    k::FusePlan F = k::fuse_plan(fs.nf, fs.ns, fs.parent, fs.by_height[0], fs.by_height[1], k::kFuseSmemCap);
    if (F.par.empty()) return;
    L.fuse_n = (int)F.par.size();
    L.fuse_n0 = (int)F.rest0.size();
    L.fuse_n1 = (int)F.rest1.size();
    L.fuse_rows = F.rows;
    L.fuse_front = F.front;
    auto nz = [](std::vector<int> &v) -> std::vector<int> & {
        if (v.empty()) v.push_back(0);
        return v;
    };
    L.fuse_par.upload(F.par, s);
    L.fuse_cptr.upload(F.cptr, s);
    L.fuse_cid.upload(nz(F.cid), s);
    L.fuse_rest0.upload(nz(F.rest0), s);
    L.fuse_rest1.upload(nz(F.rest1), s);
    HSIM_CUDA(cudaStreamSynchronize(s));  // the uploads read the host vectors
}

void build_inverse_plan(LevelData &L, cudaStream_t s) {
    const FrontSymbolic &fs = L.fs;
    k::InversePlan P = k::inverse_plan(fs.nf, fs.ns, fs.foff);
    {
        L.inv_p1_tc.clear();
        L.inv_p2_tc.clear();
        L.inv_tiles_tc.clear();
        for (size_t lv = 0; lv < P.p1.size(); ++lv) {
            std::vector<k::GemmTask> a = P.p1[lv], b = P.p2[lv];
            L.inv_tiles_tc.push_back(k::gemm_tiles_tc(a));
            k::gemm_tiles_tc(b);
            L.inv_p1_tc.emplace_back();
            L.inv_p1_tc.back().upload(a, s);
            L.inv_p2_tc.emplace_back();
            L.inv_p2_tc.back().upload(b, s);
            HSIM_CUDA(cudaStreamSynchronize(s));  // the uploads read a and b
        }
        std::vector<k::GemmTask> wt, wc;
        for (const auto &t : P.w) (t.K >= kTcMinPivots ? wt : wc).push_back(t);
        L.inv_nw_tc = (int)wt.size();
        L.inv_tw_tc = k::gemm_tiles_tc(wt);
        L.inv_nw_cc = (int)wc.size();
        L.inv_tw_cc = number_tiles(wc, k::kGemmTile);
        if (wt.empty()) wt.push_back(k::GemmTask{});
        if (wc.empty()) wc.push_back(k::GemmTask{});
        L.inv_w_tc.upload(wt, s);
        L.inv_w_cc.upload(wc, s);
        HSIM_CUDA(cudaStreamSynchronize(s));
    }
    // trailing-update tiles of the blocked factorisation
    {
        std::vector<k::SchurTask> tasks;
        L.schur_off.assign(fs.max_height + 1, {});
        constexpr int B = k::kSchurBlock;
        for (int h = 0; h <= fs.max_height; ++h) {
            int maxnf = 0, maxns = 0;
            for (int t : fs.by_height[h]) {
                maxnf = std::max(maxnf, fs.nf[t]);
                maxns = std::max(maxns, fs.ns[t]);
            }
            if (maxnf < kTcMinSchurFront) continue;
            for (int K0 = 0; K0 < maxns; K0 += B) {
                L.schur_off[h].push_back((int64_t)tasks.size());
                for (int t : fs.by_height[h]) {
                    if (fs.ns[t] <= K0 || fs.nf[t] <= K0 + B) continue;
                    const int nt = (fs.nf[t] - K0 - B + B - 1) / B;
                    for (int ti = 0; ti < nt; ++ti)
                        for (int tj = 0; tj <= ti; ++tj) tasks.push_back(k::SchurTask{t, ti * B, tj * B});
                }
            }
            L.schur_off[h].push_back((int64_t)tasks.size());
        }
        L.schur_tasks.upload(tasks.empty() ? std::vector<k::SchurTask>{k::SchurTask{}} : tasks, s);
        HSIM_CUDA(cudaStreamSynchronize(s));  // the upload reads tasks
    }
    L.n_inv_blk = (int)P.blk.size();
    L.inv_blk.upload(P.blk.empty() ? std::vector<int2>{make_int2(0, 0)} : P.blk, s);
    L.inv_p1.clear();
    L.inv_p2.clear();
    L.inv_n.clear();
    L.inv_tiles = P.tiles;
    for (size_t lv = 0; lv < P.p1.size(); ++lv) {
        L.inv_n.push_back((int)P.p1[lv].size());
        L.inv_p1.emplace_back();
        L.inv_p1.back().upload(P.p1[lv], s);
        L.inv_p2.emplace_back();
        L.inv_p2.back().upload(P.p2[lv], s);
    }
    L.inv_nw = (int)P.w.size();
    L.inv_tw = P.wtiles;
    L.inv_w.upload(P.w, s);
    L.inv_wc.upload(P.wc, s);
    L.inv_scratch = P.scratch;
    // the uploads read the host vectors of P
    HSIM_CUDA(cudaStreamSynchronize(s));
    L.h_maxnf.assign(fs.max_height + 1, 0);
    L.h_maxns.assign(fs.max_height + 1, 0);
    for (int h = 0; h <= fs.max_height; ++h)
        for (int t : fs.by_height[h]) {
            L.h_maxnf[h] = std::max(L.h_maxnf[h], fs.nf[t]);
            L.h_maxns[h] = std::max(L.h_maxns[h], fs.ns[t]);
        }
    build_fuse_plan(L, s);
}

void upload_level(LevelData &L, cudaStream_t s) {
    L.dpat.upload(L.pat_int, s);
    L.dvmap.upload(L.vmap, s);
    std::vector<int> row_of(L.pat_int.nnz());
    for (int i = 0; i < L.pat_int.n_rows; ++i)
        for (int e = L.pat_int.ptr[i]; e < L.pat_int.ptr[i + 1]; ++e) row_of[e] = i;
    L.drow_of.upload(row_of, s);
    if (L.dense) return;
    FrontSymbolic &fs = L.fs;
    L.d_foff.upload(fs.foff, s);
    L.d_rows_off.upload(fs.rows_off, s);
    L.d_relmap_off.upload(fs.relmap_off, s);
    L.d_nf.upload(fs.nf, s);
    L.d_ns.upload(fs.ns, s);
    L.d_pstart.upload(fs.pstart, s);
    L.d_rows.upload(fs.rows, s);
    L.d_relmap.upload(fs.relmap.empty() ? std::vector<int>{0} : fs.relmap, s);
    L.d_parent.upload(fs.parent, s);
    L.d_perm.upload(fs.perm, s);
    L.d_iperm.upload(fs.iperm, s);
    L.d_asm.upload(assembly_map(fs, L.pat_int), s);
    std::vector<int> hn, ea;
    L.hnodes_off.clear();
    L.ea_off.clear();
    L.step_cnt.assign(fs.max_height + 1, {});
    L.step_maxnf.assign(fs.max_height + 1, {});
    L.ea_maxu.assign(fs.max_height + 1, 0);
    for (int h = 0; h <= fs.max_height; ++h) {
        const auto &nodes = fs.by_height[h];
        L.hnodes_off.push_back((int64_t)hn.size());
        hn.insert(hn.end(), nodes.begin(), nodes.end());
        int steps = nodes.empty() ? 0 : fs.nsteps[nodes[0]];
        for (int kst = 0; kst < steps; ++kst) {
            int cnt = 0, mx = 0;
            for (int t : nodes) {
                if (fs.nsteps[t] <= kst) break;
                ++cnt;
                mx = std::max(mx, fs.nf[t]);
            }
            L.step_cnt[h].push_back(cnt);
            L.step_maxnf[h].push_back(mx);
        }
        L.ea_off.push_back((int64_t)ea.size());
        for (int c : fs.ea_children[h]) {
            ea.push_back(c);
            L.ea_maxu[h] = std::max(L.ea_maxu[h], fs.nf[c] - fs.ns[c]);
        }
    }
    L.hnodes_off.push_back((int64_t)hn.size());
    L.ea_off.push_back((int64_t)ea.size());
    L.d_hnodes.upload(hn.empty() ? std::vector<int>{0} : hn, s);
    L.d_ea.upload(ea.empty() ? std::vector<int>{0} : ea, s);
    L.fd = k::FrontDev{L.d_foff.p, L.d_nf.p, L.d_ns.p, L.d_pstart.p, L.d_rows_off.p, L.d_rows.p, L.d_relmap_off.p,
                       L.d_relmap.p};
    build_inverse_plan(L, s);
}

// Numeric LDL^T of K = S - mu M on level L (values in internal order), with
// the factor stored in precision T.  Returns the number of negative pivots
// (eigenvalues of (S, M) below mu).  Pivots below rel_tol * max|K_ii| count as
// a breakdown.
// Inverts the pivot blocks of all fronts in place and forms W = L_bs Linv
// (the inverted-factor form of k_finv.cu).
template <typename T>
void invert_level_t(cudaStream_t s, LevelData &L, T *arena, DevBuf<T> &scr) {
    scr.reserve((size_t)std::max<int64_t>(L.inv_scratch, 1));
    k::inv_diag_blocks(s, L.fd, L.inv_blk.p, L.n_inv_blk, arena);
    if constexpr (std::is_same<T, float>::value) {
        if (tc32_enabled()) {
            // block doubling: bs = 32 on the CUDA cores, 64 and up on the tensor cores
            for (size_t lv = 0; lv < L.inv_n.size(); ++lv) {
                if (lv == 0) {
                    k::gemm_tasks<T>(s, L.inv_p1[lv].p, L.inv_n[lv], L.inv_tiles[lv], arena, arena, scr.p);
                    k::gemm_tasks<T>(s, L.inv_p2[lv].p, L.inv_n[lv], L.inv_tiles[lv], arena, scr.p, arena);
                } else {
                    k::gemm_tasks_tc(s, L.inv_p1_tc[lv].p, L.inv_n[lv], L.inv_tiles_tc[lv], arena, arena, scr.p);
                    k::gemm_tasks_tc(s, L.inv_p2_tc[lv].p, L.inv_n[lv], L.inv_tiles_tc[lv], arena, scr.p, arena);
                }
            }
            k::gemm_tasks_tc(s, L.inv_w_tc.p, L.inv_nw_tc, L.inv_tw_tc, arena, arena, scr.p);
            k::gemm_tasks<T>(s, L.inv_w_cc.p, L.inv_nw_cc, L.inv_tw_cc, arena, arena, scr.p);
            k::copy_tasks<T>(s, L.inv_wc.p, L.inv_nw, L.inv_tw, scr.p, arena);
            return;
        }
    }
    for (size_t lv = 0; lv < L.inv_n.size(); ++lv) {
        k::gemm_tasks<T>(s, L.inv_p1[lv].p, L.inv_n[lv], L.inv_tiles[lv], arena, arena, scr.p);
        k::gemm_tasks<T>(s, L.inv_p2[lv].p, L.inv_n[lv], L.inv_tiles[lv], arena, scr.p, arena);
    }
    k::gemm_tasks<T>(s, L.inv_w.p, L.inv_nw, L.inv_tw, arena, arena, scr.p);
    k::copy_tasks<T>(s, L.inv_wc.p, L.inv_nw, L.inv_tw, scr.p, arena);
}

template <typename T>
int factor_level_t(hsim_ctx *ctx, LevelData &L, const double *S, const double *M, const double *Md, double mu,
                   DevBuf<T> &arena, DevBuf<T> &dpos, DevBuf<T> &dinv, DevBuf<T> &scr, double rel_tol) {
    cudaStream_t s = ctx->stream;
    FrontSymbolic &fs = L.fs;
    arena.reserve((size_t)fs.arena);
    dpos.reserve((size_t)L.n);
    HSIM_CUDA(cudaMemsetAsync(arena.p, 0, (size_t)fs.arena * sizeof(T), s));
    k::front_assemble(s, L.dpat.nnz, L.drow_of.p, L.dpat.col.p, L.d_asm.p, S, M, Md, mu, arena.p);
    unsigned long long *mx = ctx->scratch_u64.p;
    HSIM_CUDA(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s));
    k::front_maxdiag(s, L.fd, fs.n_nodes, (const T *)arena.p, mx);
    unsigned long long hmx = 0;
    HSIM_CUDA(cudaMemcpyAsync(&hmx, mx, sizeof(hmx), cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaStreamSynchronize(s));
    double maxdiag;
    std::memcpy(&maxdiag, &hmx, sizeof(double));
    const double tol = std::max(rel_tol * maxdiag, 1e-300);
    int *flags = ctx->flags.p;
    HSIM_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), s));
    for (int h = 0; h <= fs.max_height; ++h) {
        const int *nodes = L.d_hnodes.p + L.hnodes_off[h];
        int nea = (int)(L.ea_off[h + 1] - L.ea_off[h]);
        if (nea > 0) k::front_extend_add(s, L.fd, L.d_parent.p, L.d_ea.p + L.ea_off[h], nea, L.ea_maxu[h], arena.p);
        // FP32 fronts of the largest heights: blocks of kSchurBlock columns,
        // the panels' updates restricted to the block, then the block's
        // trailing update on the tensor cores; otherwise panel by panel
        const bool blocked = std::is_same<T, float>::value && tc32_enabled() && !L.schur_off[h].empty();
        constexpr int spb = k::kSchurBlock / kPanel;  // panels per block
        for (size_t kst = 0; kst < L.step_cnt[h].size(); ++kst) {
            int cnt = L.step_cnt[h][kst];
            int k0 = (int)kst * kPanel;
            int mrows = L.step_maxnf[h][kst] - k0 - 1;
            k::front_panel(s, L.fd, nodes, cnt, k0, mrows, arena.p, tol, flags);
            const int K0 = (int)(kst / spb) * k::kSchurBlock;
            k::front_update(s, L.fd, nodes, cnt, k0, mrows, arena.p, blocked ? K0 + k::kSchurBlock : INT_MAX);
            const bool block_end = (kst + 1) % spb == 0 || kst + 1 == L.step_cnt[h].size();
            if (blocked && block_end) {
                const size_t b = kst / spb;
                const int64_t t0 = L.schur_off[h][b], t1 = L.schur_off[h][b + 1];
                k::schur_tc(s, L.fd, L.schur_tasks.p + t0, (int)(t1 - t0), K0, reinterpret_cast<float *>(arena.p));
            }
        }
    }
    // all nodes 0..N-1 are listed in d_hnodes grouped by height
    k::front_diag(s, L.fd, L.d_hnodes.p, fs.n_nodes, (const T *)arena.p, dpos.p, flags + 2);
    if (std::is_same<T, float>::value) {
        // FP32 factors are solved in the inverted form (see solve_level_t)
        dinv.reserve((size_t)L.n);
        k::reciprocal(s, L.n, (const T *)dpos.p, dinv.p);
        invert_level_t<T>(s, L, arena.p, scr);
    }
    HSIM_CUDA(cudaMemcpyAsync(ctx->hflags.data(), flags, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaStreamSynchronize(s));
    if (ctx->hflags[0] != 0)
        fail(HSIM_E_BREAKDOWN, "LDL^T breakdown: " + std::to_string(ctx->hflags[0]) +
                                   " pivot(s) below tolerance (shift " + std::to_string(mu) + ")");
    return ctx->hflags[2];
}

// K^-1 X in place with the factor walked panel by panel: per tree height the
// fused kernels for fronts of one panel, else a triangle and an update launch
// per 32-column panel; then D^-1; then the backward sweep.
template <typename T>
void solve_level_panels(hsim_ctx *ctx, LevelData &L, const T *arena, const T *dpos, T *X, int k, int ldx) {
    cudaStream_t s = ctx->stream;
    const FrontSymbolic &fs = L.fs;
    auto small = [&](int h) { return L.step_cnt[h].size() == 1 && L.step_maxnf[h][0] <= k::kSmallNf; };
    for (int h = 0; h <= fs.max_height; ++h) {
        const int *nodes = L.d_hnodes.p + L.hnodes_off[h];
        if (small(h)) {
            k::solve_fwd_small(s, L.fd, nodes, L.step_cnt[h][0], L.step_maxnf[h][0], arena, k, X, ldx);
        } else {
            for (size_t kst = 0; kst < L.step_cnt[h].size(); ++kst) {
                int cnt = L.step_cnt[h][kst];
                int k0 = (int)kst * kPanel;
                k::solve_fwd_tri(s, L.fd, nodes, cnt, k0, arena, k, X, ldx);
                k::solve_fwd_upd(s, L.fd, nodes, cnt, k0, L.step_maxnf[h][kst] - k0 - 1, arena, k, X, ldx);
            }
        }
    }
    k::solve_diag(s, L.n, k, dpos, X, ldx);
    for (int h = fs.max_height; h >= 0; --h) {
        const int *nodes = L.d_hnodes.p + L.hnodes_off[h];
        if (small(h)) {
            k::solve_bwd_small(s, L.fd, nodes, L.step_cnt[h][0], L.step_maxnf[h][0], arena, k, X, ldx);
        } else {
            for (int kst = (int)L.step_cnt[h].size() - 1; kst >= 0; --kst) {
                int cnt = L.step_cnt[h][kst];
                int k0 = kst * kPanel;
                k::solve_bwd_upd(s, L.fd, nodes, cnt, k0, L.step_maxnf[h][kst] - k0 - 1, arena, k, X, ldx);
                k::solve_bwd_tri(s, L.fd, nodes, cnt, k0, arena, k, X, ldx);
            }
        }
    }
}

// K^-1 X in place (X: n x k, leading dimension ldx, internal order).
// FP32 factors are in the inverted form: one forward product per tree height
// upwards, one backward product per height downwards (k_finv.cu), Y holding
// the forward result.  FP64 factors are solved panel by panel (k_front.cu):
// at the FP64 rate of this GPU the inverted form's extra work on the
// triangular blocks costs more than the launch chains it removes.
template <typename T>
void solve_level_t(hsim_ctx *ctx, LevelData &L, const T *arena, const T *dpos, const T *dinv, DevBuf<T> &Y, T *X,
                   int k, int ldx) {
    cudaStream_t s = ctx->stream;
    const FrontSymbolic &fs = L.fs;
    if (!std::is_same<T, float>::value) {
        solve_level_panels(ctx, L, arena, dpos, X, k, ldx);
        return;
    }
    Y.reserve((size_t)L.n * ldx);
    // HSIM_TRACE=2: time of every tree height of the forward and backward sweeps
    const bool detail = trace_level() >= 2;
    std::vector<cudaEvent_t> ev;
    auto mark = [&] {
        if (!detail) return;
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        ev.push_back(e);
    };
    mark();
    const bool fused = L.fuse_n > 0 && fuse_enabled();
    for (int h = 0; h <= fs.max_height; ++h) {
        const int *nodes = L.d_hnodes.p + L.hnodes_off[h];
        const int cnt = (int)(L.hnodes_off[h + 1] - L.hnodes_off[h]);
        if constexpr (std::is_same<T, float>::value) {
            if (fused && h <= 1) {
                // leaves of unfused parents first, then the fused fronts with
                // their leaves; the unfused fronts of height 1 after both
                if (h == 0) {
                    k::solve_fwd_inv(s, L.fd, L.fuse_rest0.p, L.fuse_n0, L.h_maxnf[0], L.h_maxns[0], arena, k, X,
                                     Y.p, ldx);
                    k::solve_fwd_fused(s, L.fd, L.fuse_par.p, L.fuse_n, L.fuse_cptr.p, L.fuse_cid.p, L.fuse_rows,
                                       L.fuse_front, arena, dinv, k, X, Y.p, ldx);
                } else {
                    k::solve_fwd_inv(s, L.fd, L.fuse_rest1.p, L.fuse_n1, L.h_maxnf[1], L.h_maxns[1], arena, k, X,
                                     Y.p, ldx);
                }
                mark();
                continue;
            }
        }
        if constexpr (std::is_same<T, float>::value) {
            if (tc32_enabled() && L.h_maxns[h] >= kTcMinFwdPivots)
                k::solve_fwd_tc(s, L.fd, nodes, cnt, L.h_maxnf[h], arena, k, X, Y.p, ldx);
            else
                k::solve_fwd_inv(s, L.fd, nodes, cnt, L.h_maxnf[h], L.h_maxns[h], arena, k, X, Y.p, ldx);
        } else {
            k::solve_fwd_inv(s, L.fd, nodes, cnt, L.h_maxnf[h], L.h_maxns[h], arena, k, X, Y.p, ldx);
        }
        mark();
    }
    mark();  // the diagonal is applied inside the backward products
    for (int h = fs.max_height; h >= 0; --h) {
        const int *nodes = L.d_hnodes.p + L.hnodes_off[h];
        const int cnt = (int)(L.hnodes_off[h + 1] - L.hnodes_off[h]);
        if constexpr (std::is_same<T, float>::value) {
            if (fused && h <= 1) {
                // the unfused fronts of height 1 and the fused fronts with
                // their leaves, then the leaves of unfused parents
                if (h == 1) {
                    k::solve_bwd_inv(s, L.fd, L.fuse_rest1.p, L.fuse_n1, L.h_maxns[1], arena, dinv, k, X, Y.p, ldx);
                    k::solve_bwd_fused(s, L.fd, L.fuse_par.p, L.fuse_n, L.fuse_cptr.p, L.fuse_cid.p, L.fuse_rows,
                                       L.fuse_front, arena, k, X, Y.p, ldx);
                } else {
                    k::solve_bwd_inv(s, L.fd, L.fuse_rest0.p, L.fuse_n0, L.h_maxns[0], arena, dinv, k, X, Y.p, ldx);
                }
                mark();
                continue;
            }
        }
        k::solve_bwd_inv(s, L.fd, nodes, cnt, L.h_maxns[h], arena, dinv, k, X, Y.p, ldx);
        mark();
    }
    if (detail) {
        cudaEventSynchronize(ev.back());
        const int H = fs.max_height + 1;
        std::string line = "[hsim] solve n=" + std::to_string(L.n) + " rhs=" + std::to_string(k);
        if (fused)
            line += " fused " + std::to_string(L.fuse_n) + " height-1 fronts (unfused: " + std::to_string(L.fuse_n0) +
                    " leaves, " + std::to_string(L.fuse_n1) + " height-1 fronts)";
        line += " fwd/bwd ms per height:";
        for (int h = 0; h < H; ++h) {
            float a = 0, b = 0;
            cudaEventElapsedTime(&a, ev[h], ev[h + 1]);
            cudaEventElapsedTime(&b, ev[2 * H - h], ev[2 * H - h + 1]);
            // flops of one direction: ns^2 (unit-lower Linv) + 2 (nf - ns) ns per column
            double gf = 0.0;
            for (int t : fs.by_height[h]) gf += ((double)fs.ns[t] * fs.ns[t] + 2.0 * (fs.nf[t] - fs.ns[t]) * fs.ns[t]) * k;
            line += " h" + std::to_string(h) + "(" + std::to_string(L.hnodes_off[h + 1] - L.hnodes_off[h]) +
                    " fronts, nf<=" + std::to_string(L.h_maxnf[h]) + ", " + std::to_string(gf * 1e-9).substr(0, 5) +
                    " GF) " + std::to_string(a).substr(0, 5) + "/" + std::to_string(b).substr(0, 5);
        }
        std::fprintf(stderr, "%s\n", line.c_str());
        for (auto e : ev) cudaEventDestroy(e);
    }
}

int factor_level(hsim_ctx *ctx, hsim_hier *H, LevelData &L, const double *S, const double *M, const double *Md,
                 double mu) {
    return factor_level_t<double>(ctx, L, S, M, Md, mu, H->arena, H->dpos, H->dinvf, H->invs, 1e-13);
}

void solve_level(hsim_ctx *ctx, hsim_hier *H, LevelData &L, double *X, int k, int ldx) {
    solve_level_t<double>(ctx, L, H->arena.p, H->dpos.p, H->dinvf.p, H->ysol, X, k, ldx);
}

int subspace_q(int p, const hsim_options &o) {
    if (o.q > 0) return o.q;
    return std::max((int)std::ceil(1.5 * p), p + 8);
}

struct Timer {
    cudaStream_t s;
    cudaEvent_t a{}, b{};
    explicit Timer(cudaStream_t st) : s(st) {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
    }
    double stop() {
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        cudaEventRecord(a, s);
        return ms;
    }
    ~Timer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

// level 0 carries the lumped (diagonal) mass unless the hierarchy was built
// with the consistent one
bool consistent_mass(const hsim_hier *H) { return H->opts.mass == HSIM_MASS_CONSISTENT; }

// M Y on level tau: diagonal at tau = 0 (lumped mass), CSR otherwise
void apply_M(hsim_ctx *ctx, hsim_hier *H, int tau, int k, const double *X, int ldx, double *Y, int ldy) {
    LevelData &L = H->lev[tau];
    if (tau == 0 && !consistent_mass(H))
        k::diag_scale(ctx->stream, L.n, k, H->Md0int.p, X, ldx, Y, ldy);
    else
        k::spmm(ctx->stream, L.n, L.dpat.ptr.p, L.dpat.col.p, tau == 0 ? H->M0int.p : H->Mv[tau].p, k, X, ldx, Y,
                ldy);
}
void apply_S(hsim_ctx *ctx, hsim_hier *H, int tau, int k, const double *X, int ldx, double *Y, int ldy) {
    LevelData &L = H->lev[tau];
    const double *v = tau == 0 ? H->S0int.p : H->Sv[tau].p;
    k::spmm(ctx->stream, L.n, L.dpat.ptr.p, L.dpat.col.p, v, k, X, ldx, Y, ldy);
}

// Rayleigh-Ritz on q x q reduced matrices; throws on failure
// lowest m (<= 0: all q) Ritz pairs of the q x q problem
// tc: transforms as FP64-accurate tensor-core products (mixed path)
void ritz_step(hsim_ctx *ctx, hsim_hier *H, int q, const double *Sbar, const double *Mbar, double *lam, double *X,
               int ldx, int *sweeps, int m, bool tc) {
    H->ritz_work.reserve(k::ritz_work_size(q));
    int rc = k::ritz(ctx->stream, q, Sbar, q, Mbar, q, lam, X, ldx, H->ritz_work.p, sweeps, ctx->flags.p,
                     ctx->hflags.data(), m, tc);
    if (rc != 0) fail(HSIM_E_NOT_SPD, "reduced mass matrix is not positive definite (q = " + std::to_string(q) + ")");
}

// Plain SIM's initial basis (Sec. 3.2, initialisation heuristic) in the
// level-0 internal order: column 0 = diag(M), columns 1..q-2 = unit vectors at
// the q - 2 smallest k_ii / m_ii (ascending, the lower vertex first on ties),
// column q - 1 = random_column(seed) (natural order, then permuted).
// Expects H->Md0int filled.
void initial_basis(hsim_ctx *ctx, hsim_hier *H, int q, uint64_t seed, const double *S_val, const double *M_diag,
                   double *Phi) {
    cudaStream_t s = ctx->stream;
    LevelData &L = H->lev[0];
    const int n = L.n;
    const Csr &A = L.pat_nat;  // S_val follows this pattern
    std::vector<int64_t> dpos(n);
    for (int i = 0; i < n; ++i) {
        auto b = A.col.begin() + A.ptr[i], e = A.col.begin() + A.ptr[i + 1];
        auto it = std::lower_bound(b, e, i);
        if (it == e || *it != i) fail(HSIM_E_INTERNAL, "level-0 pattern without a diagonal entry");
        dpos[i] = it - A.col.begin();
    }
    DevBuf<int64_t> d_dpos;
    d_dpos.upload(dpos, s);
    DevBuf<double> d_sdiag((size_t)n);
    k::gather_values(s, n, d_dpos.p, S_val, d_sdiag.p);
    std::vector<double> sd(n), md(n);
    HSIM_CUDA(cudaMemcpyAsync(sd.data(), d_sdiag.p, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaMemcpyAsync(md.data(), M_diag, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaStreamSynchronize(s));
    std::vector<int> unit_pos;
    std::vector<double> rci;
    plain_basis(n, sd.data(), md.data(), L.fs.perm.data(), L.fs.iperm.data(), q, seed, &unit_pos, &rci);
    HSIM_CUDA(cudaMemsetAsync(Phi, 0, (size_t)n * q * sizeof(double), s));
    k::copy_matrix(s, n, 1, H->Md0int.p, 1, Phi, q);
    DevBuf<double> d_rc;
    d_rc.upload(rci, s);
    k::copy_matrix(s, n, 1, d_rc.p, 1, Phi + (q - 1), q);
    std::vector<double> ones(unit_pos.size(), 1.0);
    for (size_t c = 0; c < unit_pos.size(); ++c)
        HSIM_CUDA(cudaMemcpyAsync(Phi + (size_t)unit_pos[c] * q + 1 + c, &ones[c], sizeof(double),
                                  cudaMemcpyHostToDevice, s));
    HSIM_CUDA(cudaStreamSynchronize(s));  // before the host and scratch buffers go
}

void run_solve(hsim_ctx *ctx, hsim_hier *H, const double *S_val, const double *M_diag, int p, double tol,
               const hsim_options &o, double *evals, double *evecs, hsim_info *info) {
    cudaStream_t s = ctx->stream;
    Timer tm(s), total(s);
    hsim_info inf{};
    const int T = H->T;
    inf.levels = T;
    for (int t = 0; t < T && t < 8; ++t) inf.sizes[t] = H->sizes[t];
    const int q = subspace_q(p, o);
    HSIM_CHECK_ARG(q >= p && q <= H->sizes[T - 1], "subspace size q exceeds the coarsest level");
    inf.q = q;
    // plain SIM (a hierarchy built with plain_sim): Alg. 1 on the only level
    // from the initialisation heuristic, FP64
    const bool plain = H->opts.plain_sim != 0;
    HSIM_CHECK_ARG(!plain || o.precision == HSIM_FP64, "plain SIM runs in FP64 only");
    LevelData &L0 = H->lev[0];
    const int n0 = L0.n;
    // level-0 values in internal order
    H->S0int.reserve(L0.dpat.nnz);
    H->Md0int.reserve(n0);
    H->dinv0.reserve(n0);
    k::gather_values(s, L0.dpat.nnz, L0.dvmap.p, S_val, H->S0int.p);
    const bool cm = consistent_mass(H);
    if (cm) {
        // consistent M^0 in S's pattern; its row sums are the lumped mass M_L,
        // whose inverse bounds the M^-1-norms of the convergence test
        H->M0int.reserve(L0.dpat.nnz);
        k::gather_values(s, L0.dpat.nnz, L0.dvmap.p, M_diag, H->M0int.p);
        k::row_sums(s, n0, L0.dpat.ptr.p, H->M0int.p, H->Md0int.p);
    } else if (T > 1 || !L0.dense) {
        k::gather_values_i(s, n0, L0.dense ? nullptr : L0.d_perm.p, M_diag, H->Md0int.p);
    }
    H->Sv.resize(T);
    H->Mv.resize(T);
    // Galerkin products (Alg. 3, restriction step)
    for (int tau = 0; tau + 1 < T; ++tau) {
        ProlongData &P = H->pro[tau];
        LevelData &Lf = H->lev[tau];
        LevelData &Lc = H->lev[tau + 1];
        H->tval_s.reserve(P.T_pat.nnz());
        H->tval_m.reserve(P.T_pat.nnz());
        const double *Sf = tau == 0 ? H->S0int.p : H->Sv[tau].p;
        k::galerkin_au(s, Lf.n, Lf.dpat.ptr.p, Lf.dpat.col.p, Sf, P.dU.ptr.p, P.dU.col.p, P.dUval.p, P.dT.ptr.p,
                       P.dT.col.p, H->tval_s.p);
        if (tau == 0 && !cm)
            k::galerkin_au(s, Lf.n, H->d_diag_ptr.p, H->d_diag_col.p, H->Md0int.p, P.dU.ptr.p, P.dU.col.p, P.dUval.p,
                           P.dT.ptr.p, P.dT.col.p, H->tval_m.p);
        else
            k::galerkin_au(s, Lf.n, Lf.dpat.ptr.p, Lf.dpat.col.p, tau == 0 ? H->M0int.p : H->Mv[tau].p, P.dU.ptr.p,
                           P.dU.col.p, P.dUval.p, P.dT.ptr.p, P.dT.col.p, H->tval_m.p);
        H->Sv[tau + 1].reserve(Lc.dpat.nnz);
        H->Mv[tau + 1].reserve(Lc.dpat.nnz);
        k::galerkin_utt(s, Lc.n, P.dUt.ptr.p, P.dUt.col.p, P.dUtval.p, P.dT.ptr.p, P.dT.col.p, H->tval_s.p,
                        Lc.dpat.ptr.p, Lc.dpat.col.p, H->Sv[tau + 1].p);
        k::galerkin_utt(s, Lc.n, P.dUt.ptr.p, P.dUt.col.p, P.dUtval.p, P.dT.ptr.p, P.dT.col.p, H->tval_m.p,
                        Lc.dpat.ptr.p, Lc.dpat.col.p, H->Mv[tau + 1].p);
    }
    inf.ms_galerkin = tm.stop();
    // coarsest level: dense generalised eigenproblem (Alg. 3)
    LevelData &Lc = H->lev[T - 1];
    const int nc = Lc.n;
    std::vector<double> lam_h(q);
    int sweeps = 0;
    if (!plain) {
        H->Sbar.reserve((size_t)nc * nc);
        H->Mbar.reserve((size_t)nc * nc);
        if (T == 1) {
            k::densify(s, nc, Lc.dpat.ptr.p, Lc.dpat.col.p, H->S0int.p, H->Sbar.p);
            if (cm) k::densify(s, nc, Lc.dpat.ptr.p, Lc.dpat.col.p, H->M0int.p, H->Mbar.p);
            else k::densify_diag(s, nc, M_diag, H->Mbar.p);
        } else {
            k::densify(s, nc, Lc.dpat.ptr.p, Lc.dpat.col.p, H->Sv[T - 1].p, H->Sbar.p);
            k::densify(s, nc, Lc.dpat.ptr.p, Lc.dpat.col.p, H->Mv[T - 1].p, H->Mbar.p);
        }
        H->coarseX.reserve((size_t)nc * nc);
        H->coarseLam.reserve(nc);
        ritz_step(ctx, H, nc, H->Sbar.p, H->Mbar.p, H->coarseLam.p, H->coarseX.p, nc, &sweeps, q,
                  o.precision == HSIM_MIXED);
        inf.coarse_sweeps = sweeps;
        inf.ms_coarse = tm.stop();
        HSIM_CUDA(cudaMemcpyAsync(lam_h.data(), H->coarseLam.p, q * sizeof(double), cudaMemcpyDeviceToHost, s));
        HSIM_CUDA(cudaStreamSynchronize(s));
    }
    H->signs.reserve(std::max(p, 1));
    if (T == 1 && !plain) {
        HSIM_CUDA(cudaMemcpyAsync(evals, H->coarseLam.p, p * sizeof(double), cudaMemcpyDeviceToDevice, s));
        k::output_evecs(s, nc, p, nullptr, H->coarseX.p, nc, evecs, H->signs.p);
        HSIM_CUDA(cudaStreamSynchronize(s));
        inf.ms_total = total.stop();
        if (info) *info = inf;
        return;
    }
    // SIM on every finer level
    const size_t nq = (size_t)n0 * q;
    H->Phi.reserve(nq);
    H->Psi.reserve(nq);
    H->SP.reserve(nq);
    H->MP.reserve(nq);
    H->Sbar.reserve((size_t)q * q);
    H->Mbar.reserve((size_t)q * q);
    H->phibar.reserve((size_t)q * q);
    H->lam.reserve(q);
    H->colw.reserve(q);
    H->res_sums.reserve(3 * (size_t)q);
    const double *Xc = H->coarseX.p;
    int ldxc = nc;
    std::vector<double> rs(3 * (size_t)q), res(q);
    for (int tau = plain ? 0 : T - 2; tau >= 0; --tau) {
        LevelData &L = H->lev[tau];
        const int n = L.n;
        Timer tp(s);
        if (plain) {
            initial_basis(ctx, H, q, o.seed, S_val, M_diag, H->Phi.p);
        } else {
            // prolongation of the basis (Alg. 3)
            ProlongData &P = H->pro[tau];
            k::spmm(s, n, P.dU.ptr.p, P.dU.col.p, P.dUval.p, q, Xc, ldxc, H->Phi.p, q);
        }
        inf.ms_prolong += tp.stop();
        // shift (Alg. 3): Lambda_j of the coarser level, j = floor(alpha p); for
        // j = 0 mirrored below zero to -lambda_ref so that S - mu M stays away
        // from the constant null vector.  Plain SIM: the given shift (Alg. 1).
        int j = (int)std::floor(o.alpha * p);
        double mu = plain ? o.sim_shift : lam_h[j];
        if (!plain && j == 0) {
            mu = -lam_h[q - 1];
            for (int i = 0; i < q; ++i)
                if (lam_h[i] > 1e-8 * lam_h[q - 1]) {
                    mu = -lam_h[i];
                    break;
                }
        }
        // Mixed precision factors K in FP32.  The pivot-free LDL^T of an
        // indefinite K shows element growth near 5e4 (an FP32 factor is then
        // only ~3e-3 accurate), so the mixed path shifts below the spectrum,
        // mu = -max(lambda_ref, 0.01 Lambda_{q-1}): K is positive definite,
        // the factorisation is stable, and the convergence ratio of the top
        // pairs, (lambda_i - mu) / (lambda_q - mu), changes by about 1 %.
        const bool mixed = o.precision == HSIM_MIXED;
        const int q32 = (q + 3) & ~3;  // FP32 block rows 16-byte aligned (vector atomics)
        if (mixed) {
            double lam_ref = lam_h[q - 1];
            for (int i = 0; i < q; ++i)
                if (lam_h[i] > 1e-8 * lam_h[q - 1]) {
                    lam_ref = lam_h[i];
                    break;
                }
            mu = -std::max(lam_ref, 0.01 * lam_h[q - 1]);
        }
        inf.shift[tau] = mu;
        const double *Sx = tau == 0 ? H->S0int.p : H->Sv[tau].p;
        const double *Mx = tau == 0 ? (cm ? H->M0int.p : nullptr) : H->Mv[tau].p;
        const double *Mdx = (tau == 0 && !cm) ? H->Md0int.p : nullptr;
        Timer tf(s);
        int negp = mixed ? factor_level_t<float>(ctx, L, Sx, Mx, Mdx, mu, H->arena32, H->dpos32, H->dinvf32, H->invs32, 1e-7)
                         : factor_level(ctx, H, L, Sx, Mx, Mdx, mu);
        inf.ms_factor += tf.stop();
        if (mixed) {
            if (negp != 0)
                fail(HSIM_E_BREAKDOWN, "FP32 factor of the positive definite shifted matrix has " +
                                           std::to_string(negp) + " negative pivot(s)");
            H->X32.reserve((size_t)n * q32);
            H->rho.reserve(3 * (size_t)q);
        }
        // One inverse iteration in correction form (mixed path): for any
        // scalar rho, K^-1 M psi = (psi - K^-1 (S psi - rho M psi)) / (rho - mu).
        // With rho the Rayleigh quotient the right-hand side is the residual,
        // small next to psi, so the FP32 solve's error is small next to the
        // FP64 psi it corrects; the factor 1 / (rho - mu) > 0 is dropped (the
        // columns are rescaled before the Gram).  X, SX, MX: FP64, columns
        // [0, a) with leading dimension q; num / den give rho per column.
        // MX == nullptr: M is the diagonal Md0int (level 0) and M X is not formed
        auto correction_step = [&](const double *X, const double *SX, const double *MX, const double *num,
                                   const double *den, double *Y, int a) {
            if (MX) k::residual_f32(s, n, a, SX, q, MX, q, num, den, H->rho.p + 2 * q, H->X32.p, q32);
            else k::residual_f32_diag(s, n, a, SX, q, X, q, H->Md0int.p, num, den, H->rho.p + 2 * q, H->X32.p, q32);
            solve_level_t<float>(ctx, L, H->arena32.p, H->dpos32.p, H->dinvf32.p, H->ysol32, H->X32.p, a, q32);
            k::sub_f2d(s, n, a, X, q, H->X32.p, q32, Y, q);
        };
        if (trace_on())
            std::fprintf(stderr, "[hsim] level %d n=%d q=%d shift=%.10g negative_pivots=%d fronts=%d nnzL=%lld\n", tau,
                         n, q, mu, negp, L.fs.n_nodes, (long long)L.fs.nnz_L);
        inf.factor_nnz[tau] = L.fs.nnz_L;
        inf.factor_flops[tau] = L.fs.flops;
        // 1 / diag(M) for the M^-1 norm of the finest level (Sec. 5, termination
        // criterion); with the consistent M, 1 / diag(M_L) of the lumped mass and
        // twice the resulting ratio (M_L / 4 <= M <= M_L bounds the exact norms)
        const double norm_bound = (tau == 0 && cm) ? 2.0 : 1.0;
        const double *dinv = nullptr;
        if (tau == 0) {
            H->dinv0.reserve(n);
            k::reciprocal(s, n, H->Md0int.p, H->dinv0.p);
            dinv = H->dinv0.p;
        }
        // M Phi
        apply_M(ctx, H, tau, q, H->Phi.p, q, H->MP.p, q);
        int locked = 0, it = 0;
        double maxres = 0.0, prev_maxres = 0.0;
        // The shifted matrix is factored without pivoting; element growth can
        // leave a backward error well above the unit roundoff, which puts a
        // floor under the residual.  One step of FP64 refinement of the last
        // inverse iteration removes it; in automatic mode it is switched on
        // once a level's residual stops decreasing.
        bool refine = o.refine > 0;
        for (it = 1; it <= o.max_iters; ++it) {
            const int a = q - locked;
            Timer ts(s);
            // inverse iterations on the active columns (Alg. 1, solve step; twice)
            if (mixed) {
                // first: the current Ritz pairs (S Phi, M Phi and Lambda from the
                // last convergence test; at it = 1 Phi is the prolonged basis,
                // whose Rayleigh quotients are the coarse Ritz values)
                if (it == 1) apply_S(ctx, H, tau, a, H->Phi.p + locked, q, H->SP.p + locked, q);
                const double *lam_d = (it == 1 && tau == T - 2) ? H->coarseLam.p : H->lam.p;
                correction_step(H->Phi.p + locked, H->SP.p + locked, H->MP.p + locked, lam_d + locked, nullptr,
                                H->Psi.p + locked, a);
                for (int extra = 1; extra < o.inv_iters; ++extra) {
                    double *Pa = H->Psi.p + locked;
                    apply_S(ctx, H, tau, a, Pa, q, H->SP.p + locked, q);
                    if (tau == 0 && !cm) {
                        // diagonal M: M Psi enters only through m_i psi_i (MP is
                        // recomputed for the Gram below)
                        k::col_dots2_diag_mixed(s, n, a, Pa, q, H->SP.p + locked, q, H->Md0int.p, H->rho.p,
                                                H->rho.p + q);
                        correction_step(Pa, H->SP.p + locked, nullptr, H->rho.p, H->rho.p + q, Pa, a);
                    } else {
                        apply_M(ctx, H, tau, a, Pa, q, H->MP.p + locked, q);
                        k::col_dots2_mixed(s, n, a, Pa, q, H->SP.p + locked, H->MP.p + locked, q, H->rho.p,
                                           H->rho.p + q);
                        correction_step(Pa, H->SP.p + locked, H->MP.p + locked, H->rho.p, H->rho.p + q, Pa, a);
                    }
                }
            } else {
                k::copy_matrix(s, n, a, H->MP.p + locked, q, H->Psi.p + locked, q);
                solve_level(ctx, H, L, H->Psi.p + locked, a, q);
                for (int extra = 1; extra < o.inv_iters; ++extra) {
                    apply_M(ctx, H, tau, a, H->Psi.p + locked, q, H->SP.p + locked, q);
                    k::copy_matrix(s, n, a, H->SP.p + locked, q, H->Psi.p + locked, q);
                    solve_level(ctx, H, L, H->Psi.p + locked, a, q);
                }
            }
            if (refine && !mixed) {
                // right-hand side of the last solve: SP (two or more inverse
                // iterations) or MP (one); the residual goes to the other buffer
                double *rhs = o.inv_iters >= 2 ? H->SP.p : H->MP.p;
                double *res_buf = o.inv_iters >= 2 ? H->MP.p : H->SP.p;
                k::shifted_residual(s, n, L.dpat.ptr.p, L.dpat.col.p, Sx, Mx, Mdx, mu, a, H->Psi.p + locked, q,
                                    rhs + locked, q, res_buf + locked, q);
                solve_level(ctx, H, L, res_buf + locked, a, q);
                k::axpy_matrix(s, n, a, res_buf + locked, q, H->Psi.p + locked, q);
            }
            if (locked > 0) k::copy_matrix(s, n, locked, H->Phi.p, q, H->Psi.p, q);
            inf.solve_flops += 4.0 * (double)L.fs.nnz_L * a * (o.inv_iters + ((refine && !mixed) ? 1 : 0));
            double ph[6];
            inf.ms_solve += (ph[0] = ts.stop());
            // S Psi, M Psi (Alg. 1, reduced matrices).  The columns of Psi are
            // scaled to unit M-norm on the q x q side: with W = diag(M_bar)^-1/2,
            // S_bar = W Psi^T S Psi W, M_bar = W Psi^T M Psi W and Phi = Psi (W Phi_bar).
            // The locked columns of Psi are copies of Phi's, whose S Phi and
            // M Phi from the last convergence test are still in SP and MP (the
            // inverse iterations write columns >= locked only): only the
            // active columns are multiplied.
            apply_M(ctx, H, tau, q - locked, H->Psi.p + locked, q, H->MP.p + locked, q);
            apply_S(ctx, H, tau, q - locked, H->Psi.p + locked, q, H->SP.p + locked, q);
            inf.ms_spmm += (ph[1] = ts.stop());
            if (mixed) {
                // Grams on BF16 tensor cores, Psi split once.  Gram errors rotate the
                // Ritz basis inside span(Psi) (the subspace itself is unaffected) and
                // add about E / lambda_i to the residual of pair i: five digits
                // (2^-39 of the column maxima) leave ~1e-8 at lambda_q / lambda_1 ~ 10^3,
                // enough below tolerances of 1e-6 and up; tighter ones take six.
                const int gd = tol >= kGramFiveDigitTol ? 5 : 6;
                const size_t part = k::ozaki_cols_scratch(n, q);
                H->oz.reserve(3 * part);
                k::OzakiOperand X = k::ozaki_split_cols(s, n, q, H->Psi.p, q, H->oz.p, gd);
                k::OzakiOperand YS = k::ozaki_split_cols(s, n, q, H->SP.p, q, H->oz.p + part, gd);
                k::OzakiOperand YM = k::ozaki_split_cols(s, n, q, H->MP.p, q, H->oz.p + 2 * part, gd);
                const double t_split = ts.stop();
                k::ozaki_product(s, X, YS, X.kp, H->Sbar.p, q, 0, true);
                k::ozaki_product(s, X, YM, X.kp, H->Mbar.p, q, 0, true);
                const double t_prod = ts.stop();
                inf.ms_tc_product += t_prod;
                ph[2] = t_split + t_prod;
            } else {
                k::gram(s, n, q, q, H->Psi.p, q, H->SP.p, q, H->Sbar.p, q, true);
                k::gram(s, n, q, q, H->Psi.p, q, H->MP.p, q, H->Mbar.p, q, true);
            }
            k::scale_sym_unit_diag(s, q, H->Sbar.p, H->Mbar.p, q, H->colw.p);
            if (mixed) inf.ms_gram += (ph[2] += ts.stop());
            else inf.ms_gram += (ph[2] = ts.stop());
            // dense eigenproblem (Alg. 1): Ritz values ascending, M-orthonormal
            ritz_step(ctx, H, q, H->Sbar.p, H->Mbar.p, H->lam.p, H->phibar.p, q, &sweeps, 0, mixed);
            inf.ritz_calls += 1;
            inf.ritz_sweeps += sweeps;
            k::diag_scale(s, q, q, H->colw.p, H->phibar.p, q, H->phibar.p, q);  // W Phi_bar
            inf.ms_ritz += (ph[3] = ts.stop());
            // update Phi = Psi Phi_bar (Alg. 1)
            if (mixed) {
                const size_t part = k::ozaki_rows_scratch(n, q);
                H->oz.reserve(part + k::ozaki_cols_scratch(q, q));
                k::OzakiOperand X = k::ozaki_split_rows(s, n, q, H->Psi.p, q, H->oz.p);
                k::OzakiOperand Y = k::ozaki_split_cols(s, q, q, H->phibar.p, q, H->oz.p + part);
                const double t_split = ts.stop();
                k::ozaki_product(s, X, Y, X.kp, H->Phi.p, q, 1);
                const double t_prod = ts.stop();
                inf.ms_tc_product += t_prod;
                ph[4] = t_split + t_prod;
            } else {
                k::gemm_nn(s, n, q, q, H->Psi.p, q, H->phibar.p, q, H->Phi.p, q);
            }
            if (mixed) inf.ms_update += ph[4];
            else inf.ms_update += (ph[4] = ts.stop());
            // convergence test (eq. conv2)
            apply_S(ctx, H, tau, q, H->Phi.p, q, H->SP.p, q);
            apply_M(ctx, H, tau, q, H->Phi.p, q, H->MP.p, q);
            // only the pairs i < p enter the test and the locking
            if (mixed) k::residual_sums_mixed(s, n, p, H->SP.p, q, H->MP.p, q, H->lam.p, dinv, H->res_sums.p);
            else k::residual_sums(s, n, p, H->SP.p, q, H->MP.p, q, H->lam.p, dinv, H->res_sums.p);
            HSIM_CUDA(cudaMemcpyAsync(rs.data(), H->res_sums.p, 3 * p * sizeof(double), cudaMemcpyDeviceToHost, s));
            HSIM_CUDA(cudaMemcpyAsync(lam_h.data(), H->lam.p, q * sizeof(double), cudaMemcpyDeviceToHost, s));
            HSIM_CUDA(cudaStreamSynchronize(s));
            if (mixed) {
                k::ozaki_check(s);
                k::tc32_check(s);
            }
            inf.ms_residual += (ph[5] = ts.stop());
            double lam_ref = lam_h[q - 1];
            for (int i = 0; i < q; ++i)
                if (lam_h[i] > 1e-8 * lam_h[q - 1]) {
                    lam_ref = lam_h[i];
                    break;
                }
            maxres = 0.0;
            for (int i = 0; i < p; ++i) {
                double den = std::max(std::sqrt(rs[3 * i + 1]), lam_ref * std::sqrt(rs[3 * i + 2]));
                res[i] = norm_bound * std::sqrt(rs[3 * i]) / den;
                maxres = std::max(maxres, res[i]);
            }
            if (trace_on())
                std::fprintf(stderr,
                             "[hsim] level %d it %d locked %d max_res %.3e ritz_sweeps %d refine %d lam0 %.6g lam_p %.6g"
                             " ms solve %.1f spmm %.1f gram %.1f ritz %.1f update %.1f residual %.1f\n",
                             tau, it, locked, maxres, sweeps, (int)refine, lam_h[0], lam_h[p - 1], ph[0], ph[1], ph[2],
                             ph[3], ph[4], ph[5]);
            if (!(maxres < tol) && !std::isfinite(maxres)) fail(HSIM_E_INTERNAL, "non-finite residual");
            if (maxres < tol) break;
            if (o.refine == 0 && !refine && it >= 2 && maxres > 0.7 * prev_maxres && maxres < 1e-6) refine = true;
            prev_maxres = maxres;
            int r = 0;
            while (r < p && res[r] < o.lock_factor * tol) ++r;
            locked = r;
        }
        if (it > o.max_iters) {
            inf.iters[tau] = o.max_iters;
            if (info) *info = inf;
            fail(HSIM_E_NO_CONVERGENCE, "level " + std::to_string(tau) + ": no convergence in " +
                                            std::to_string(o.max_iters) + " iterations (max residual " +
                                            std::to_string(maxres) + ")");
        }
        inf.iters[tau] = it;
        if (tau == 0) inf.max_residual = maxres;
        // the next finer level starts from this level's basis
        Xc = H->Phi.p;
        ldxc = q;
        if (tau > 0) {
            // Phi is overwritten by the prolongation on the next level: keep a copy
            H->coarseX.reserve((size_t)n * q);
            k::copy_matrix(s, n, q, H->Phi.p, q, H->coarseX.p, q);
            Xc = H->coarseX.p;
        }
    }
    HSIM_CUDA(cudaMemcpyAsync(evals, H->lam.p, p * sizeof(double), cudaMemcpyDeviceToDevice, s));
    k::output_evecs(s, n0, p, L0.d_iperm.p, H->Phi.p, q, evecs, H->signs.p);
    HSIM_CUDA(cudaStreamSynchronize(s));
    inf.ms_total = total.stop();
    if (info) *info = inf;
}

// Per directed mesh edge (entry of the mesh pattern A0), the triangle corners
// opposite it (two slots, -1 = none); every vertex's triangles (CSR).
struct AssemblyMaps {
    std::vector<int> ecot, vcount, vt;
};
AssemblyMaps assembly_maps(const Csr &A0, const int32_t *F, int n, int m) {
    AssemblyMaps am;
    am.ecot.assign(2 * (size_t)A0.nnz(), -1);
    auto find = [&](int i, int j) -> int64_t {
        auto b = A0.col.begin() + A0.ptr[i], e = A0.col.begin() + A0.ptr[i + 1];
        auto it = std::lower_bound(b, e, j);
        if (it == e || *it != j) fail(HSIM_E_INTERNAL, "mesh edge missing in pattern");
        return it - A0.col.begin();
    };
    am.vcount.assign(n + 1, 0);
    for (int t = 0; t < m; ++t)
        for (int kc = 0; kc < 3; ++kc) {
            int a = F[3 * t + (kc + 1) % 3], b = F[3 * t + (kc + 2) % 3];
            for (int64_t e : {find(a, b), find(b, a)}) {
                if (am.ecot[2 * e] < 0) am.ecot[2 * e] = 3 * t + kc;
                else if (am.ecot[2 * e + 1] < 0) am.ecot[2 * e + 1] = 3 * t + kc;
                else fail(HSIM_E_INVALID_ARG, "non-manifold edge (more than two triangles)");
            }
            am.vcount[F[3 * t + kc] + 1]++;
        }
    for (int i = 0; i < n; ++i) am.vcount[i + 1] += am.vcount[i];
    am.vt.resize(am.vcount.back());
    std::vector<int> fill(am.vcount.begin(), am.vcount.end() - 1);
    for (int t = 0; t < m; ++t)
        for (int kc = 0; kc < 3; ++kc) am.vt[fill[F[3 * t + kc]]++] = t;
    return am;
}

hsim_hier *build(hsim_ctx *ctx, int n, int m, const double *V, const int32_t *F, const double *L2, int p,
                 const hsim_options &o) {
    HSIM_CHECK_ARG(p >= 1, "p must be >= 1");
    cudaStream_t s = ctx->stream;
    auto H = std::make_unique<hsim_hier>();
    H->ctx = ctx;
    H->device = ctx->device;
    H->m = m;
    H->p = p;
    H->opts = o;
    const bool dirichlet = o.boundary == HSIM_BOUNDARY_DIRICHLET;
    const int leaf = o.leaf_size > 0 ? o.leaf_size : 32;
    // plain SIM: one sparse level (no sampling, no prolongation)
    const bool plain = o.plain_sim != 0;
    // HSIM_TRACE set: wall time of each part of the build on stderr
    auto tb = std::chrono::steady_clock::now();
    auto lap = [&](const char *what) {
        if (!trace_on()) return;
        const auto t1 = std::chrono::steady_clock::now();
        std::fprintf(stderr, "[hsim] hierarchy build: %s %.1f ms\n", what,
                     std::chrono::duration<double, std::milli>(t1 - tb).count());
        tb = t1;
    };
    HostHierarchy hh =
        host_levels(n, m, V, F, L2, p, plain ? 1 : o.levels, o.start_vertex, o.sigma, subspace_q(p, o), dirichlet);
    lap("mesh graph, level-0 pattern, sizes");
    // the assembly maps need only the mesh: built on a worker thread while the
    // hierarchy is sampled (joined before the uploads)
    std::future<AssemblyMaps> fam =
        std::async(std::launch::async, [&hh, F, n, m] { return assembly_maps(hh.A_mesh, F, n, m); });
    H->sizes = hh.sizes;
    const int T = (int)H->sizes.size();
    H->T = T;
    H->n_mesh = n;
    H->n = H->sizes[0];
    H->lev.resize(T);
    H->pro.resize(T - 1);
    H->lev[0].n = H->n;
    H->lev[0].pat_nat = std::move(hh.A0);
    // the symbolic analysis of level 0 needs only its pattern: it runs on a
    // worker thread while the sampling and the prolongations are built (the
    // future is declared after H, so it is joined before H is released)
    std::future<FrontSymbolic> fs0;
    if (T > 1) fs0 = std::async(std::launch::async, [&H, leaf] { return analyse(H->lev[0].pat_nat, leaf); });
    if (o.hier_device) device_samples(hh, V, o.start_vertex, o.sigma, s);
    else host_samples(hh, o.start_vertex, o.sigma);
    lap(o.hier_device ? "sampling and prolongations (GPU)" : "sampling and prolongations (host)");
    H->order = std::move(hh.order);
    const Csr &Amesh = hh.A_mesh;  // every mesh edge plus the diagonal
    if (dirichlet) {
        H->d_smap.upload(hh.smap, s);
        H->d_dofs.upload(hh.dofs, s);
        H->dofs = std::move(hh.dofs);
    }
    for (int tau = 0; tau + 1 < T; ++tau) {
        ProlongData &P = H->pro[tau];
        P.U_nat = std::move(hh.U[tau]);
        P.rho = hh.rho[tau];
        P.fallback = hh.fallback[tau];
        Csr Ut = transpose_pattern(P.U_nat);
        Csr AU = pattern_product(H->lev[tau].pat_nat, P.U_nat);
        H->lev[tau + 1].n = H->sizes[tau + 1];
        H->lev[tau + 1].pat_nat = pattern_product(Ut, AU);
    }
    lap("Galerkin patterns");
    // orderings and symbolic analyses
    for (int tau = T - 1; tau >= 0; --tau) {
        LevelData &L = H->lev[tau];
        L.dense = (tau == T - 1) && !plain;
        if (!L.dense) {
            L.fs = (tau == 0 && fs0.valid()) ? fs0.get() : analyse(L.pat_nat, leaf);
        } else {
            L.fs.n = L.n;
            L.fs.perm.resize(L.n);
            L.fs.iperm.resize(L.n);
            for (int i = 0; i < L.n; ++i) L.fs.perm[i] = L.fs.iperm[i] = i;
        }
        L.pat_int = permute_symmetric(L.pat_nat, L.fs.iperm, &L.vmap);
    }
    for (int tau = 0; tau + 1 < T; ++tau) {
        ProlongData &P = H->pro[tau];
        P.U_int = permute_rows_cols(P.U_nat, H->lev[tau].fs.iperm, H->lev[tau + 1].fs.iperm);
        P.Ut_int = transpose_pattern(P.U_int);
        P.T_pat = pattern_product(H->lev[tau].pat_int, P.U_int);
        Csr C = pattern_product(P.Ut_int, P.T_pat);
        if (C.ptr != H->lev[tau + 1].pat_int.ptr || C.col != H->lev[tau + 1].pat_int.col)
            fail(HSIM_E_INTERNAL, "Galerkin pattern mismatch between orders");
    }
    lap("orderings and symbolic analyses (level 0 joined)");
    // device uploads
    for (int tau = 0; tau < T; ++tau) upload_level(H->lev[tau], s);
    for (int tau = 0; tau + 1 < T; ++tau) {
        ProlongData &P = H->pro[tau];
        P.dU.upload(P.U_int, s);
        P.dUval.upload(P.U_int.val, s);
        P.dUt.upload(P.Ut_int, s);
        P.dUtval.upload(P.Ut_int.val, s);
        P.dT.upload(P.T_pat, s);
    }
    {
        const int n0 = H->n;  // the level-0 mass matrix is diagonal: identity pattern
        std::vector<int> dp(n0 + 1), dc(n0);
        for (int i = 0; i <= n0; ++i) dp[i] = i;
        for (int i = 0; i < n0; ++i) dc[i] = i;
        H->d_diag_ptr.upload(dp, s);
        H->d_diag_col.upload(dc, s);
    }
    // level-0 assembly data in the natural pattern of the whole mesh
    const Csr &A0 = Amesh;
    H->pat0.upload(H->lev[0].pat_nat, s);
    if (dirichlet) H->patm.upload(A0, s);
    AssemblyMaps am = fam.get();
    std::vector<int> &ecot = am.ecot, &vcount = am.vcount, &vt = am.vt;
    std::vector<int> Fv(F, F + 3 * (size_t)m);
    H->d_ecot.upload(ecot, s);
    H->d_vt_ptr.upload(vcount, s);
    H->d_vt_idx.upload(vt, s);
    H->dF.upload(Fv, s);
    HSIM_CUDA(cudaStreamSynchronize(s));
    lap("uploads and assembly maps");
    return H.release();
}

hsim_options checked(const hsim_options *o) {
    hsim_options d;
    hsim_default_options(&d);
    if (!o) return d;
    hsim_options r = *o;
    HSIM_CHECK_ARG(r.sigma > 0, "sigma must be positive");
    HSIM_CHECK_ARG(r.alpha >= 0 && r.alpha < 1, "alpha must be in [0, 1)");
    HSIM_CHECK_ARG(r.max_iters >= 1, "max_iters must be >= 1");
    HSIM_CHECK_ARG(r.inv_iters >= 1, "inv_iters must be >= 1");
    HSIM_CHECK_ARG(r.precision == HSIM_FP64 || r.precision == HSIM_MIXED, "unknown precision");
    HSIM_CHECK_ARG(r.refine >= -1 && r.refine <= 1, "refine must be -1, 0 or 1");
    HSIM_CHECK_ARG(r.boundary == HSIM_BOUNDARY_NATURAL || r.boundary == HSIM_BOUNDARY_DIRICHLET,
                   "unknown boundary condition");
    HSIM_CHECK_ARG(r.plain_sim == 0 || r.plain_sim == 1, "plain_sim must be 0 or 1");
    HSIM_CHECK_ARG(std::isfinite(r.sim_shift), "sim_shift must be finite");
    HSIM_CHECK_ARG(r.mass == HSIM_MASS_LUMPED || r.mass == HSIM_MASS_CONSISTENT, "unknown mass matrix");
    HSIM_CHECK_ARG(r.plain_sim == 0 || r.mass == HSIM_MASS_LUMPED, "plain SIM takes the lumped mass matrix");
    HSIM_CHECK_ARG(r.hier_device == 0 || r.hier_device == 1, "hier_device must be 0 or 1");
    return r;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void hsim_default_options(hsim_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->levels = 0;
    o->sigma = 7.0;
    o->alpha = 0.1;
    o->max_iters = 100;
    o->inv_iters = 2;
    o->lock_factor = 0.1;
    o->precision = HSIM_FP64;
    o->start_vertex = 0;
    o->leaf_size = 32;
    o->q = 0;
    o->refine = 0;
    o->boundary = HSIM_BOUNDARY_NATURAL;
    o->plain_sim = 0;
    o->sim_shift = 0.0;
    o->seed = 0;
    o->mass = HSIM_MASS_LUMPED;
    o->hier_device = 1;
}

void hsim_random_column(int n, uint64_t seed, double *out) {
    if (n > 0 && out) random_column(n, seed, out);
}

const char *hsim_last_error(void) { return g_last_error.c_str(); }

uint64_t hsim_kernel_launches(void) { return g_launches.load(); }

hsim_status hsim_create(int device, void *stream, hsim_ctx **out) {
    return guard([&] {
        HSIM_CHECK_ARG(out != nullptr, "out is NULL");
        int count = 0;
        HSIM_CUDA(cudaGetDeviceCount(&count));
        HSIM_CHECK_ARG(device >= 0 && device < count, "no such CUDA device");
        DeviceGuard dg(device);
        auto c = std::make_unique<hsim_ctx>();
        c->device = device;
        c->stream = (cudaStream_t)stream;
        c->flags.alloc(16);
        c->hflags.assign(16, 0);
        c->scratch_u64.alloc(4);
        *out = c.release();
    });
}

void hsim_destroy(hsim_ctx *ctx) {
    if (!ctx) return;
    // never throws: at process exit the CUDA runtime may already be gone
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    delete ctx;
    if (prev >= 0) cudaSetDevice(prev);
    cudaGetLastError();
}

hsim_status hsim_build_hierarchy(hsim_ctx *ctx, int n, int m, const double *V, const int32_t *F, const double *L2,
                                 int p, const hsim_options *opts, hsim_hier **out) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx && out, "NULL argument");
        DeviceGuard dg(ctx->device);
        hsim_options o = checked(opts);
        HSIM_CHECK_ARG(o.start_vertex >= 0 && o.start_vertex < n, "start_vertex out of range");
        *out = build(ctx, n, m, V, F, L2, p, o);
    });
}

void hsim_hier_destroy(hsim_hier *h) {
    if (!h) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    delete h;
    if (prev >= 0) cudaSetDevice(prev);
    cudaGetLastError();
}

hsim_status hsim_hier_info(const hsim_hier *h, int *levels, int *sizes, int32_t *order) {
    return guard([&] {
        HSIM_CHECK_ARG(h, "NULL hierarchy");
        if (levels) *levels = h->T;
        if (sizes)
            for (int t = 0; t < h->T && t < 8; ++t) sizes[t] = h->sizes[t];
        if (order && !h->order.empty()) std::memcpy(order, h->order.data(), h->order.size() * sizeof(int32_t));
    });
}

hsim_status hsim_hier_dofs(const hsim_hier *h, int32_t *dofs) {
    return guard([&] {
        HSIM_CHECK_ARG(h && dofs, "NULL argument");
        if (h->dofs.empty())
            for (int i = 0; i < h->n; ++i) dofs[i] = i;
        else
            std::memcpy(dofs, h->dofs.data(), h->dofs.size() * sizeof(int32_t));
    });
}

hsim_status hsim_hier_pattern(const hsim_hier *h, int *n, int64_t *nnz, const int32_t **ptr, const int32_t **col) {
    return guard([&] {
        HSIM_CHECK_ARG(h, "NULL hierarchy");
        if (n) *n = h->n;
        if (nnz) *nnz = h->pat0.nnz;
        if (ptr) *ptr = h->pat0.ptr.p;
        if (col) *col = h->pat0.col.p;
    });
}

hsim_status hsim_hier_prolongation(const hsim_hier *h, int tau, int *rows, int *cols, int64_t *nnz, int32_t *ptr,
                                   int32_t *col, double *val) {
    return guard([&] {
        HSIM_CHECK_ARG(h && tau >= 0 && tau + 1 < h->T, "bad level");
        const Csr &U = h->pro[tau].U_nat;
        if (rows) *rows = U.n_rows;
        if (cols) *cols = U.n_cols;
        if (nnz) *nnz = U.nnz();
        if (ptr) std::memcpy(ptr, U.ptr.data(), U.ptr.size() * sizeof(int));
        if (col) std::memcpy(col, U.col.data(), U.col.size() * sizeof(int));
        if (val) std::memcpy(val, U.val.data(), U.val.size() * sizeof(double));
    });
}

hsim_status hsim_assemble(hsim_ctx *ctx, const hsim_hier *h, const double *V_dev, const double *L2_dev,
                          double *S_val, double *M_diag) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx && h && S_val && M_diag, "NULL argument");
        HSIM_CHECK_ARG((V_dev != nullptr) != (L2_dev != nullptr), "exactly one of V and L2 must be given");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"V", V_dev}, {"L2", L2_dev}, {"S_val", S_val}, {"M_diag", M_diag}});
        cudaStream_t s = ctx->stream;
        DevBuf<double> cot((size_t)3 * h->m), area((size_t)h->m), Sm, Mm;
        const bool cm = consistent_mass(h);
        k::triangle_geometry(s, h->m, h->dF.p, V_dev, L2_dev, cot.p, area.p);
        if (h->dofs.empty()) {
            k::assemble_sm(s, h->n, h->pat0.ptr.p, h->pat0.col.p, h->d_ecot.p, cot.p, h->d_vt_ptr.p, h->d_vt_idx.p,
                           area.p, S_val, M_diag, cm);
        } else {
            // Dirichlet: the whole mesh, then the interior rows and columns
            Sm.alloc((size_t)h->patm.nnz);
            Mm.alloc(cm ? (size_t)h->patm.nnz : (size_t)h->n_mesh);
            k::assemble_sm(s, h->n_mesh, h->patm.ptr.p, h->patm.col.p, h->d_ecot.p, cot.p, h->d_vt_ptr.p,
                           h->d_vt_idx.p, area.p, Sm.p, Mm.p, cm);
            k::gather_values(s, h->pat0.nnz, h->d_smap.p, Sm.p, S_val);
            if (cm) k::gather_values(s, h->pat0.nnz, h->d_smap.p, Mm.p, M_diag);
            else k::gather_values_i(s, h->n, h->d_dofs.p, Mm.p, M_diag);
        }
        HSIM_CUDA(cudaStreamSynchronize(s));  // before the temporaries are freed
    });
}

hsim_status hsim_solve(hsim_ctx *ctx, hsim_hier *h, const double *S_val, const double *M_diag, int p, double tol,
                       const hsim_options *opts, double *evals, double *evecs, hsim_info *info) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx && h && S_val && M_diag && evals && evecs, "NULL argument");
        HSIM_CHECK_ARG(p >= 1 && p <= h->n, "bad p");
        HSIM_CHECK_ARG(tol > 0, "tol must be positive");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"S_val", S_val}, {"M_diag", M_diag}, {"evals", evals}, {"evecs", evecs}});
        hsim_options o = checked(opts ? opts : &h->opts);
        run_solve(ctx, h, S_val, M_diag, p, tol, o, evals, evecs, info);
    });
}

hsim_status hsim_solve_batched(hsim_ctx *ctx, int nmesh, hsim_hier *const *hiers, const double *const *S_vals,
                               const double *const *M_diags, const int *p, double tol, const hsim_options *opts,
                               double *const *evals, double *const *evecs, hsim_info *infos, int streams) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx, "NULL context");
        HSIM_CHECK_ARG(nmesh >= 0 && tol > 0, "bad nmesh or tol");
        if (nmesh == 0) return;
        HSIM_CHECK_ARG(hiers && S_vals && M_diags && p && evals && evecs, "NULL argument");
        std::set<const hsim_hier *> seen;
        for (int i = 0; i < nmesh; ++i) {
            HSIM_CHECK_ARG(hiers[i] && S_vals[i] && M_diags[i] && evals[i] && evecs[i],
                           "NULL argument for mesh " + std::to_string(i));
            HSIM_CHECK_ARG(p[i] >= 1 && p[i] <= hiers[i]->n, "bad p for mesh " + std::to_string(i));
            HSIM_CHECK_ARG(hiers[i]->device == ctx->device, "mesh " + std::to_string(i) + " lives on another device");
            // a hierarchy holds the workspace of its solve: one solve per hierarchy at a time
            HSIM_CHECK_ARG(seen.insert(hiers[i]).second, "hierarchy listed twice (mesh " + std::to_string(i) + ")");
        }
        DeviceGuard dg(ctx->device);
        for (int i = 0; i < nmesh; ++i)
            check_device_ptrs(ctx->device, {{"S_vals[i]", S_vals[i]}, {"M_diags[i]", M_diags[i]},
                                            {"evals[i]", evals[i]}, {"evecs[i]", evecs[i]}});
        const int W = std::max(1, std::min(nmesh, streams > 0 ? streams : 8));
        // inputs produced on the caller's stream are complete before any worker starts
        cudaEvent_t ready;
        HSIM_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        std::vector<std::unique_ptr<hsim_ctx>> wctx;
        auto cleanup = [&] {
            for (auto &c : wctx)
                if (c && c->stream) {
                    cudaStreamSynchronize(c->stream);
                    cudaStreamDestroy(c->stream);
                    c->stream = nullptr;
                }
            cudaEventDestroy(ready);
        };
        try {
            HSIM_CUDA(cudaEventRecord(ready, ctx->stream));
            for (int w = 0; w < W; ++w) {
                auto c = std::make_unique<hsim_ctx>();
                c->device = ctx->device;
                HSIM_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
                c->flags.alloc(16);
                c->hflags.assign(16, 0);
                c->scratch_u64.alloc(4);
                HSIM_CUDA(cudaStreamWaitEvent(c->stream, ready, 0));
                wctx.push_back(std::move(c));
            }
        } catch (...) {
            cleanup();
            throw;
        }
        // workers take meshes from a shared counter, largest first (a large
        // mesh started last would set the batch's tail); the first error
        // stops the others before their next mesh
        std::vector<int> order(nmesh);
        for (int i = 0; i < nmesh; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hiers[a]->n > hiers[b]->n; });
        std::atomic<int> next{0};
        std::atomic<bool> stop{false};
        std::mutex emu;
        hsim_status status = HSIM_OK;
        std::string message;
        auto record = [&](hsim_status st, int i, const std::string &m) {
            std::lock_guard<std::mutex> lock(emu);
            if (status == HSIM_OK) {
                status = st;
                message = "mesh " + std::to_string(i) + ": " + m;
            }
            stop = true;
        };
        std::vector<std::thread> pool;
        for (int w = 0; w < W; ++w) {
            pool.emplace_back([&, w] {
                if (cudaSetDevice(ctx->device) != cudaSuccess) {
                    record(HSIM_E_CUDA, -1, "cudaSetDevice failed in a worker");
                    return;
                }
                for (;;) {
                    if (stop) break;
                    const int k = next.fetch_add(1);
                    if (k >= nmesh) break;
                    const int i = order[k];
                    try {
                        hsim_options o = checked(opts ? opts : &hiers[i]->opts);
                        run_solve(wctx[w].get(), hiers[i], S_vals[i], M_diags[i], p[i], tol, o, evals[i], evecs[i],
                                  infos ? &infos[i] : nullptr);
                    } catch (const Error &e) {
                        record(e.status, i, e.what());
                    } catch (const std::bad_alloc &) {
                        record(HSIM_E_NOMEM, i, "host allocation failed");
                    } catch (const std::exception &e) {
                        record(HSIM_E_INTERNAL, i, e.what());
                    }
                }
            });
        }
        for (auto &t : pool) t.join();
        cleanup();
        if (status != HSIM_OK) fail(status, message);
    });
}

hsim_status hsim_eig_grad(hsim_ctx *ctx, int n, int m, const double *V, const int32_t *F, int p,
                          const double *evals, const double *evecs, const double *dloss, double *dV) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx, "NULL context");
        HSIM_CHECK_ARG(n >= 0 && m >= 0 && p >= 0, "bad sizes");
        if (n == 0) return;
        HSIM_CHECK_ARG(V && dV && (m == 0 || F), "NULL argument");
        HSIM_CHECK_ARG(p == 0 || (evals && evecs && dloss), "NULL argument");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"V", V}, {"F", F}, {"evals", evals}, {"evecs", evecs}, {"dloss", dloss},
                                        {"dV", dV}});
        k::eig_grad(ctx->stream, n, p == 0 ? 0 : m, p, V, F, evals, evecs, n, dloss, dV);
        HSIM_CUDA(cudaStreamSynchronize(ctx->stream));
    });
}

hsim_status hsim_spmm(hsim_ctx *ctx, int n_rows, int n_cols, const int32_t *ptr, const int32_t *col,
                      const double *val, int k, const double *X, int ldx, double *Y, int ldy) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx, "NULL context");
        HSIM_CHECK_ARG(n_rows >= 0 && n_cols >= 0 && k >= 0 && ldx >= k && ldy >= k, "bad sizes");
        if (n_rows == 0 || k == 0) return;
        HSIM_CHECK_ARG(ptr && col && X && Y && (val || n_cols == 0), "NULL argument");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"row_ptr", ptr}, {"col", col}, {"val", val}, {"X", X}, {"Y", Y}});
        k::spmm(ctx->stream, n_rows, ptr, col, val, k, X, ldx, Y, ldy);
        HSIM_CUDA(cudaStreamSynchronize(ctx->stream));
    });
}

hsim_status hsim_gram(hsim_ctx *ctx, int n, int ka, int kb, const double *A, int lda, const double *B, int ldb,
                      double *G) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx && A && B && G, "NULL argument");
        HSIM_CHECK_ARG(n >= 0 && ka >= 0 && kb >= 0 && lda >= ka && ldb >= kb, "bad sizes");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"A", A}, {"B", B}, {"G", G}});
        k::gram(ctx->stream, n, ka, kb, A, lda, B, ldb, G, kb, false);
        HSIM_CUDA(cudaStreamSynchronize(ctx->stream));
    });
}

hsim_status hsim_gemm_update(hsim_ctx *ctx, int n, int kk, int m, const double *A, int lda, const double *B, int ldb,
                             double *C, int ldc) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx && A && B && C, "NULL argument");
        HSIM_CHECK_ARG(n >= 0 && kk >= 0 && m >= 0 && lda >= kk && ldb >= m && ldc >= m, "bad sizes");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"A", A}, {"B", B}, {"C", C}});
        k::gemm_nn(ctx->stream, n, kk, m, A, lda, B, ldb, C, ldc);
        HSIM_CUDA(cudaStreamSynchronize(ctx->stream));
    });
}

hsim_status hsim_gram_tc(hsim_ctx *ctx, int n, int ka, int kb, const double *A, int lda, const double *B, int ldb,
                         double *G, int digits) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx && A && B && G, "NULL argument");
        HSIM_CHECK_ARG(n >= 1 && ka >= 1 && kb >= 1 && lda >= ka && ldb >= kb, "bad sizes");
        HSIM_CHECK_ARG(digits == 5 || digits == 6, "digits must be 5 or 6");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"A", A}, {"B", B}, {"G", G}});
        DevBuf<unsigned char> scratch(k::ozaki_cols_scratch(n, ka) + k::ozaki_cols_scratch(n, kb));
        k::OzakiOperand X = k::ozaki_split_cols(ctx->stream, n, ka, A, lda, scratch.p, digits);
        k::OzakiOperand Y =
            k::ozaki_split_cols(ctx->stream, n, kb, B, ldb, scratch.p + k::ozaki_cols_scratch(n, ka), digits);
        k::ozaki_product(ctx->stream, X, Y, X.kp, G, kb, 0);
        k::ozaki_check(ctx->stream);
    });
}

hsim_status hsim_gemm_update_tc(hsim_ctx *ctx, int n, int kk, int m, const double *A, int lda, const double *B,
                                int ldb, double *C, int ldc) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx && A && B && C, "NULL argument");
        HSIM_CHECK_ARG(n >= 1 && kk >= 1 && m >= 1 && lda >= kk && ldb >= m && ldc >= m, "bad sizes");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"A", A}, {"B", B}, {"C", C}});
        DevBuf<unsigned char> scratch(k::ozaki_rows_scratch(n, kk) + k::ozaki_cols_scratch(kk, m));
        k::OzakiOperand X = k::ozaki_split_rows(ctx->stream, n, kk, A, lda, scratch.p);
        k::OzakiOperand Y = k::ozaki_split_cols(ctx->stream, kk, m, B, ldb, scratch.p + k::ozaki_rows_scratch(n, kk));
        k::ozaki_product(ctx->stream, X, Y, X.kp, C, ldc, 1);
        k::ozaki_check(ctx->stream);
    });
}

namespace {
hsim_status ritz_entry(hsim_ctx *ctx, int kk, const double *Sbar, const double *Mbar, double *evals, double *X,
                       int *sweeps_out, bool tc) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx && Sbar && Mbar && evals && X, "NULL argument");
        HSIM_CHECK_ARG(kk >= 1, "bad size");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"Sbar", Sbar}, {"Mbar", Mbar}, {"evals", evals}, {"X", X}});
        DevBuf<double> work(k::ritz_work_size(kk));
        int sw = 0;
        int rc = k::ritz(ctx->stream, kk, Sbar, kk, Mbar, kk, evals, X, kk, work.p, &sw, ctx->flags.p,
                         ctx->hflags.data(), 0, tc);
        HSIM_CUDA(cudaStreamSynchronize(ctx->stream));
        if (sweeps_out) *sweeps_out = sw;
        if (rc != 0) fail(HSIM_E_NOT_SPD, "M_bar is not positive definite");
    });
}
}  // namespace

hsim_status hsim_ritz(hsim_ctx *ctx, int kk, const double *Sbar, const double *Mbar, double *evals, double *X,
                      int *sweeps_out) {
    return ritz_entry(ctx, kk, Sbar, Mbar, evals, X, sweeps_out, false);
}

hsim_status hsim_ritz_tc(hsim_ctx *ctx, int kk, const double *Sbar, const double *Mbar, double *evals, double *X,
                         int *sweeps_out) {
    return ritz_entry(ctx, kk, Sbar, Mbar, evals, X, sweeps_out, true);
}

hsim_status hsim_galerkin(hsim_ctx *ctx, int n, int nc, const int32_t *A_ptr, const int32_t *A_col,
                          const double *A_val, const int32_t *U_ptr, const int32_t *U_col, const double *U_val,
                          int64_t *nnz_out, int32_t **C_ptr, int32_t **C_col, double **C_val) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx && A_ptr && A_col && A_val && U_ptr && U_col && U_val && nnz_out && C_ptr && C_col && C_val,
                       "NULL argument");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"A_val", A_val}, {"U_val", U_val}});
        cudaStream_t s = ctx->stream;
        Csr A, U;
        A.n_rows = A.n_cols = n;
        A.ptr.assign(A_ptr, A_ptr + n + 1);
        A.col.assign(A_col, A_col + A.ptr[n]);
        U.n_rows = n;
        U.n_cols = nc;
        U.ptr.assign(U_ptr, U_ptr + n + 1);
        U.col.assign(U_col, U_col + U.ptr[n]);
        for (int c : A.col) HSIM_CHECK_ARG(c >= 0 && c < n, "A column out of range");
        for (int c : U.col) HSIM_CHECK_ARG(c >= 0 && c < nc, "U column out of range");
        // U^T pattern with a map to U's entries
        Csr Ut;
        Ut.n_rows = nc;
        Ut.n_cols = n;
        Ut.ptr.assign(nc + 1, 0);
        for (int c : U.col) Ut.ptr[c + 1]++;
        for (int i = 0; i < nc; ++i) Ut.ptr[i + 1] += Ut.ptr[i];
        Ut.col.resize(U.col.size());
        std::vector<int> map(U.col.size());
        std::vector<int> fill(Ut.ptr.begin(), Ut.ptr.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int e = U.ptr[i]; e < U.ptr[i + 1]; ++e) {
                int d = fill[U.col[e]]++;
                Ut.col[d] = i;
                map[d] = e;
            }
        Csr Tp = pattern_product(A, U);
        Csr Cp = pattern_product(Ut, Tp);
        DevCsr dA, dU, dUt, dT;
        dA.upload(A, s);
        dU.upload(U, s);
        dUt.upload(Ut, s);
        dT.upload(Tp, s);
        DevBuf<int> dmap;
        dmap.upload(map, s);
        DevBuf<double> utv(map.size()), tv((size_t)Tp.nnz());
        k::gather_values_i(s, (int64_t)map.size(), dmap.p, U_val, utv.p);
        k::galerkin_au(s, n, dA.ptr.p, dA.col.p, A_val, dU.ptr.p, dU.col.p, U_val, dT.ptr.p, dT.col.p, tv.p);
        int32_t *cp = nullptr, *cc = nullptr;
        double *cv = nullptr;
        HSIM_CUDA(cudaMalloc(&cp, (nc + 1) * sizeof(int32_t)));
        HSIM_CUDA(cudaMalloc(&cc, std::max<int64_t>(1, Cp.nnz()) * sizeof(int32_t)));
        HSIM_CUDA(cudaMalloc(&cv, std::max<int64_t>(1, Cp.nnz()) * sizeof(double)));
        HSIM_CUDA(cudaMemcpyAsync(cp, Cp.ptr.data(), (nc + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        if (Cp.nnz())
            HSIM_CUDA(cudaMemcpyAsync(cc, Cp.col.data(), Cp.nnz() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        k::galerkin_utt(s, nc, dUt.ptr.p, dUt.col.p, utv.p, dT.ptr.p, dT.col.p, tv.p, cp, cc, cv);
        HSIM_CUDA(cudaStreamSynchronize(s));
        *nnz_out = Cp.nnz();
        *C_ptr = cp;
        *C_col = cc;
        *C_val = cv;
    });
}

void hsim_free(void *p) {
    if (p) cudaFree(p);
}

hsim_status hsim_level_pattern(const hsim_hier *h, int tau, int *n, int64_t *nnz, int32_t *ptr, int32_t *col) {
    return guard([&] {
        HSIM_CHECK_ARG(h && tau >= 0 && tau < h->T, "bad level");
        const Csr &A = h->lev[tau].pat_nat;
        if (n) *n = A.n_rows;
        if (nnz) *nnz = A.nnz();
        if (ptr) std::memcpy(ptr, A.ptr.data(), A.ptr.size() * sizeof(int));
        if (col) std::memcpy(col, A.col.data(), A.col.size() * sizeof(int));
    });
}

hsim_status hsim_shifted_solve(hsim_ctx *ctx, hsim_hier *h, int tau, const double *S_val, const double *M_val,
                               double mu, int kk, double *B, int ldb, int *neg) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx && h && S_val && M_val && B, "NULL argument");
        HSIM_CHECK_ARG(tau >= 0 && tau < h->T && !h->lev[tau].dense, "level has no sparse factorisation");
        HSIM_CHECK_ARG(kk >= 1 && ldb >= kk, "bad sizes");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"S_val", S_val}, {"M_val", M_val}, {"B", B}});
        cudaStream_t s = ctx->stream;
        LevelData &L = h->lev[tau];
        const bool diag_m = tau == 0 && !consistent_mass(h);  // M_val: n diagonal values, else S's pattern
        DevBuf<double> Sv((size_t)L.dpat.nnz), Mv(diag_m ? (size_t)L.n : (size_t)L.dpat.nnz);
        k::gather_values(s, L.dpat.nnz, L.dvmap.p, S_val, Sv.p);
        if (diag_m) k::gather_values_i(s, L.n, L.d_perm.p, M_val, Mv.p);
        else k::gather_values(s, L.dpat.nnz, L.dvmap.p, M_val, Mv.p);
        int negp = factor_level(ctx, h, L, Sv.p, diag_m ? nullptr : Mv.p, diag_m ? Mv.p : nullptr, mu);
        DevBuf<double> X((size_t)L.n * kk);
        k::gather_rows(s, L.n, kk, L.d_perm.p, B, ldb, X.p, kk);
        solve_level(ctx, h, L, X.p, kk, kk);
        k::gather_rows(s, L.n, kk, L.d_iperm.p, X.p, kk, B, ldb);
        HSIM_CUDA(cudaStreamSynchronize(s));
        k::tc32_check(s);
        if (neg) *neg = negp;
    });
}

hsim_status hsim_shifted_solve_f32(hsim_ctx *ctx, hsim_hier *h, int tau, const double *S_val, const double *M_val,
                                   double mu, int kk, double *B, int ldb, int *neg) {
    return guard([&] {
        HSIM_CHECK_ARG(ctx && h && S_val && M_val && B, "NULL argument");
        HSIM_CHECK_ARG(tau >= 0 && tau < h->T && !h->lev[tau].dense, "level has no sparse factorisation");
        HSIM_CHECK_ARG(kk >= 1 && ldb >= kk, "bad sizes");
        DeviceGuard dg(ctx->device);
        check_device_ptrs(ctx->device, {{"S_val", S_val}, {"M_val", M_val}, {"B", B}});
        cudaStream_t s = ctx->stream;
        LevelData &L = h->lev[tau];
        const bool diag_m = tau == 0 && !consistent_mass(h);  // M_val: n diagonal values, else S's pattern
        DevBuf<double> Sv((size_t)L.dpat.nnz), Mv(diag_m ? (size_t)L.n : (size_t)L.dpat.nnz);
        k::gather_values(s, L.dpat.nnz, L.dvmap.p, S_val, Sv.p);
        if (diag_m) k::gather_values_i(s, L.n, L.d_perm.p, M_val, Mv.p);
        else k::gather_values(s, L.dpat.nnz, L.dvmap.p, M_val, Mv.p);
        int negp = factor_level_t<float>(ctx, L, Sv.p, diag_m ? nullptr : Mv.p, diag_m ? Mv.p : nullptr, mu,
                                         h->arena32, h->dpos32, h->dinvf32, h->invs32, 1e-7);
        DevBuf<double> X((size_t)L.n * kk);
        k::gather_rows(s, L.n, kk, L.d_perm.p, B, ldb, X.p, kk);
        const int ld = (kk + 3) & ~3;  // 16-byte rows (vector atomics of the forward products)
        DevBuf<float> X32((size_t)L.n * ld);
        k::convert_matrix(s, L.n, kk, X.p, kk, X32.p, ld);
        solve_level_t<float>(ctx, L, h->arena32.p, h->dpos32.p, h->dinvf32.p, h->ysol32, X32.p, kk, ld);
        k::convert_matrix(s, L.n, kk, X32.p, ld, X.p, kk);
        k::gather_rows(s, L.n, kk, L.d_iperm.p, X.p, kk, B, ldb);
        HSIM_CUDA(cudaStreamSynchronize(s));
        k::tc32_check(s);
        if (neg) *neg = negp;
    });
}

}  // extern "C"
