// Host replay of the multifrontal factorisation and solve over the symbolic
// structures of host_symbolic.cpp, in the same order and with the same index
// arithmetic as the GPU kernels of k_front.cu (front arena layout, panels of
// kPanel columns, extend-add through relmap, row lists of the solves).  It
// lets the symbolic analysis be checked on a machine without a GPU; the
// solver itself never calls it.  hsim_check_inverted replays the inverted
// form of the FP32 solves (k_finv.cu) the same way: the inversion tasks of
// k::inverse_plan executed with the semantics of k_gemm_tasks, then one
// product per front and direction, optionally with heights 0 and 1 in the
// order of the fused kernels (k::fuse_plan).  hsim_check_hierarchy returns the mesh
// part of a hierarchy (level sizes, farthest-point order, prolongations) from
// the host code that hsim_build_hierarchy runs before its device uploads.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "host.h"
#include "kernels.h"

using namespace hsim;

namespace {

// Status and hsim_last_error() message of the exception being handled.
hsim_status caught() {
    try {
        throw;
    } catch (const Error &e) {
        set_last_error(e.what());
        return e.status;
    } catch (const std::bad_alloc &) {
        set_last_error("host allocation failed");
        return HSIM_E_NOMEM;
    } catch (const std::exception &e) {
        set_last_error(e.what());
        return HSIM_E_INTERNAL;
    } catch (...) {
        set_last_error("unknown error");
        return HSIM_E_INTERNAL;
    }
}

// assembly and numeric LDL^T of A over its symbolic analysis, as the GPU
// kernels do them; fills fs, the arena and the number of negative pivots
void factor_host(int n, const int32_t *ptr, const int32_t *col, const double *val, int leaf_size, FrontSymbolic &fs,
                 std::vector<double> &arena, int &neg) {
    Csr A;
    A.n_rows = A.n_cols = n;
    A.ptr.assign(ptr, ptr + n + 1);
    A.col.assign(col, col + A.ptr[n]);
    A.val.assign(val, val + A.ptr[n]);
    fs = analyse(A, leaf_size);
    std::vector<int64_t> vmap;
    Csr Ai = permute_symmetric(A, fs.iperm, &vmap);
    std::vector<int64_t> dst = assembly_map(fs, Ai);
    arena.assign(fs.arena, 0.0);
    for (int64_t e = 0; e < Ai.nnz(); ++e) {
        if (dst[e] < 0) continue;
        if (dst[e] >= fs.arena) fail(HSIM_E_INTERNAL, "assembly destination outside the arena");
        arena[dst[e]] = A.val[vmap[e]];
    }
    neg = 0;
    for (int h = 0; h <= fs.max_height; ++h) {
        for (int c : fs.ea_children[h]) {
            int p = fs.parent[c];
            int u = fs.nf[c] - fs.ns[c];
            const double *Fc = arena.data() + fs.foff[c];
            double *Fp = arena.data() + fs.foff[p];
            const int *rel = fs.relmap.data() + fs.relmap_off[c];
            for (int j = 0; j < u; ++j)
                for (int i = j; i < u; ++i) {
                    int64_t di = (int64_t)rel[j] * fs.nf[p] + rel[i];
                    if (rel[i] < rel[j] || di >= (int64_t)fs.nf[p] * fs.nf[p])
                        fail(HSIM_E_INTERNAL, "extend-add outside the parent's lower triangle");
                    Fp[di] += Fc[(int64_t)(fs.ns[c] + j) * fs.nf[c] + fs.ns[c] + i];
                }
        }
        for (int t : fs.by_height[h]) {
            const int nf = fs.nf[t], ns = fs.ns[t];
            double *F = arena.data() + fs.foff[t];
            for (int k0 = 0; k0 < ns; k0 += kPanel) {
                int kb = std::min(kPanel, ns - k0);
                // panel: LDL^T of the diagonal block, then rows below
                for (int j = 0; j < kb; ++j) {
                    double d = F[(int64_t)(k0 + j) * nf + k0 + j];
                    for (int r = j + 1; r < kb; ++r) {
                        double l = F[(int64_t)(k0 + j) * nf + k0 + r] / d;
                        for (int c = j + 1; c <= r; ++c)
                            F[(int64_t)(k0 + c) * nf + k0 + r] -= l * d * F[(int64_t)(k0 + j) * nf + k0 + c] / d;
                    }
                    for (int r = j + 1; r < kb; ++r) F[(int64_t)(k0 + j) * nf + k0 + r] /= d;
                }
                for (int r = k0 + kb; r < nf; ++r) {
                    double x[kPanel];
                    for (int c = 0; c < kb; ++c) {
                        double v = F[(int64_t)(k0 + c) * nf + r];
                        for (int cc = 0; cc < c; ++cc) v -= x[cc] * F[(int64_t)(k0 + cc) * nf + k0 + c];
                        x[c] = v;
                    }
                    for (int c = 0; c < kb; ++c) F[(int64_t)(k0 + c) * nf + r] = x[c] / F[(int64_t)(k0 + c) * nf + k0 + c];
                }
                // trailing update
                for (int c = k0 + kb; c < nf; ++c)
                    for (int r = c; r < nf; ++r) {
                        double acc = 0.0;
                        for (int kk = 0; kk < kb; ++kk)
                            acc += F[(int64_t)(k0 + kk) * nf + r] * F[(int64_t)(k0 + kk) * nf + k0 + kk] *
                                   F[(int64_t)(k0 + kk) * nf + c];
                        F[(int64_t)c * nf + r] -= acc;
                    }
            }
            for (int i = 0; i < ns; ++i) neg += F[(int64_t)i * nf + i] < 0.0;
        }
    }
}

}  // namespace

extern "C" hsim_status hsim_check_symbolic(int n, const int32_t *ptr, const int32_t *col, const double *val,
                                           int leaf_size, int nrhs, const double *B, double *X, int *neg_pivots,
                                           int64_t *nnz_L) {
    try {
        HSIM_CHECK_ARG(n > 0 && ptr && col && val && B && X && nrhs >= 1, "bad arguments");
        FrontSymbolic fs;
        std::vector<double> arena;
        int neg = 0;
        factor_host(n, ptr, col, val, leaf_size, fs, arena, neg);
        // solve in the internal order
        std::vector<double> Y((size_t)n * nrhs);
        for (int pos = 0; pos < n; ++pos)
            std::memcpy(&Y[(size_t)pos * nrhs], &B[(size_t)fs.perm[pos] * nrhs], nrhs * sizeof(double));
        auto row = [&](int t, int r) { return fs.rows[fs.rows_off[t] + r]; };
        for (int h = 0; h <= fs.max_height; ++h)
            for (int t : fs.by_height[h]) {
                const int nf = fs.nf[t], ns = fs.ns[t], ps = fs.pstart[t];
                const double *F = arena.data() + fs.foff[t];
                for (int k0 = 0; k0 < ns; k0 += kPanel) {
                    int kb = std::min(kPanel, ns - k0);
                    for (int r = 1; r < kb; ++r)
                        for (int c = 0; c < r; ++c)
                            for (int j = 0; j < nrhs; ++j)
                                Y[(size_t)(ps + k0 + r) * nrhs + j] -=
                                    F[(int64_t)(k0 + c) * nf + k0 + r] * Y[(size_t)(ps + k0 + c) * nrhs + j];
                    for (int r = k0 + kb; r < nf; ++r) {
                        int g = row(t, r);
                        if (g < 0 || g >= n) fail(HSIM_E_INTERNAL, "front row outside the matrix");
                        for (int c = 0; c < kb; ++c)
                            for (int j = 0; j < nrhs; ++j)
                                Y[(size_t)g * nrhs + j] -= F[(int64_t)(k0 + c) * nf + r] * Y[(size_t)(ps + k0 + c) * nrhs + j];
                    }
                }
            }
        for (int t = 0; t < fs.n_nodes; ++t) {
            const double *F = arena.data() + fs.foff[t];
            for (int i = 0; i < fs.ns[t]; ++i)
                for (int j = 0; j < nrhs; ++j)
                    Y[(size_t)(fs.pstart[t] + i) * nrhs + j] /= F[(int64_t)i * fs.nf[t] + i];
        }
        for (int h = fs.max_height; h >= 0; --h)
            for (int t : fs.by_height[h]) {
                const int nf = fs.nf[t], ns = fs.ns[t], ps = fs.pstart[t];
                const double *F = arena.data() + fs.foff[t];
                int nst = (ns + kPanel - 1) / kPanel;
                for (int st = nst - 1; st >= 0; --st) {
                    int k0 = st * kPanel;
                    int kb = std::min(kPanel, ns - k0);
                    for (int r = k0 + kb; r < nf; ++r) {
                        int g = row(t, r);
                        for (int c = 0; c < kb; ++c)
                            for (int j = 0; j < nrhs; ++j)
                                Y[(size_t)(ps + k0 + c) * nrhs + j] -= F[(int64_t)(k0 + c) * nf + r] * Y[(size_t)g * nrhs + j];
                    }
                    for (int r = kb - 2; r >= 0; --r)
                        for (int c = r + 1; c < kb; ++c)
                            for (int j = 0; j < nrhs; ++j)
                                Y[(size_t)(ps + k0 + r) * nrhs + j] -=
                                    F[(int64_t)(k0 + r) * nf + k0 + c] * Y[(size_t)(ps + k0 + c) * nrhs + j];
                }
            }
        for (int pos = 0; pos < n; ++pos)
            std::memcpy(&X[(size_t)fs.perm[pos] * nrhs], &Y[(size_t)pos * nrhs], nrhs * sizeof(double));
        if (neg_pivots) *neg_pivots = neg;
        if (nnz_L) *nnz_L = fs.nnz_L;
        return HSIM_OK;
    } catch (...) {
        return caught();
    }
}

namespace {

// C = (+/-) A B of one inversion task, with the operand reads of k_gemm_tasks
void run_task(const k::GemmTask &tk, const double *Ab, const double *Bb, double *Cb) {
    const bool ua = tk.flags & k::kGemmAUnitLower, ub = tk.flags & k::kGemmBUnitLower;
    auto at = [&](int i, int kk) {
        if (!ua) return Ab[tk.a + (int64_t)kk * tk.lda + i];
        return i > kk ? Ab[tk.a + (int64_t)kk * tk.lda + i] : (i == kk ? 1.0 : 0.0);
    };
    auto bt = [&](int kk, int j) {
        if (!ub) return Bb[tk.b + (int64_t)j * tk.ldb + kk];
        return kk > j ? Bb[tk.b + (int64_t)j * tk.ldb + kk] : (kk == j ? 1.0 : 0.0);
    };
    const double sg = (tk.flags & k::kGemmNeg) ? -1.0 : 1.0;
    std::vector<double> out((size_t)tk.M * tk.N);
    for (int j = 0; j < tk.N; ++j)
        for (int i = 0; i < tk.M; ++i) {
            double acc = 0.0;
            for (int kk = 0; kk < tk.K; ++kk) acc += at(i, kk) * bt(kk, j);
            out[(size_t)j * tk.M + i] = sg * acc;
        }
    for (int j = 0; j < tk.N; ++j)
        for (int i = 0; i < tk.M; ++i) Cb[tk.c + (int64_t)j * tk.ldc + i] = out[(size_t)j * tk.M + i];
}

}  // namespace

extern "C" hsim_status hsim_check_inverted(int n, const int32_t *ptr, const int32_t *col, const double *val,
                                           int leaf_size, int nrhs, const double *B, double *X, int *neg_pivots,
                                           int64_t *nnz_L, int fused_h01, int *fused_counts) {
    try {
        HSIM_CHECK_ARG(n > 0 && ptr && col && val && B && X && nrhs >= 1, "bad arguments");
        FrontSymbolic fs;
        std::vector<double> arena;
        int neg = 0;
        factor_host(n, ptr, col, val, leaf_size, fs, arena, neg);
        // inversion: 32 x 32 diagonal blocks, block-doubling levels, W = L_bs Linv
        k::InversePlan P = k::inverse_plan(fs.nf, fs.ns, fs.foff);
        for (const int2 &b : P.blk) {
            const int t = b.x, b0 = b.y, nf = fs.nf[t], kb = std::min(32, fs.ns[t] - b0);
            double *F = arena.data() + fs.foff[t];
            double Lb[32][32] = {}, Xb[32][32] = {};
            for (int r = 0; r < kb; ++r)
                for (int c = 0; c < r; ++c) Lb[r][c] = F[(int64_t)(b0 + c) * nf + b0 + r];
            for (int c = 0; c < kb; ++c) {
                Xb[c][c] = 1.0;
                for (int r = c + 1; r < kb; ++r) {
                    double acc = Lb[r][c];
                    for (int j = c + 1; j < r; ++j) acc += Lb[r][j] * Xb[j][c];
                    Xb[r][c] = -acc;
                }
            }
            for (int r = 0; r < kb; ++r)
                for (int c = 0; c < r; ++c) F[(int64_t)(b0 + c) * nf + b0 + r] = Xb[r][c];
        }
        std::vector<double> scr((size_t)std::max<int64_t>(P.scratch, 1));
        for (size_t lv = 0; lv < P.p1.size(); ++lv) {
            for (const k::GemmTask &tk : P.p1[lv]) run_task(tk, arena.data(), arena.data(), scr.data());
            for (const k::GemmTask &tk : P.p2[lv]) run_task(tk, arena.data(), scr.data(), arena.data());
        }
        for (const k::GemmTask &tk : P.w) run_task(tk, arena.data(), arena.data(), scr.data());
        for (const k::GemmTask &tk : P.wc)
            for (int j = 0; j < tk.N; ++j)
                for (int i = 0; i < tk.M; ++i)
                    arena[tk.c + (int64_t)j * tk.ldc + i] = scr[tk.a + (int64_t)j * tk.lda + i];
        std::vector<double> Xi((size_t)n * nrhs), Y((size_t)n * nrhs, 0.0);
        for (int pos = 0; pos < n; ++pos)
            std::memcpy(&Xi[(size_t)pos * nrhs], &B[(size_t)fs.perm[pos] * nrhs], nrhs * sizeof(double));
        auto row = [&](int t, int r) {
            const int g = fs.rows[fs.rows_off[t] + r];
            if (g < 0 || g >= n) fail(HSIM_E_INTERNAL, "front row outside the matrix");
            return g;
        };
        auto front = [&](int t) { return arena.data() + fs.foff[t]; };
        auto dinv = [&](int t, int r) { return 1.0 / front(t)[(int64_t)r * fs.nf[t] + r]; };
        // forward coefficient A(r, j): unit lower Linv on the pivot rows, W below
        auto fwd_a = [&](int t, int r, int j) {
            const int nf = fs.nf[t], ns = fs.ns[t];
            return (r >= ns || r > j) ? front(t)[(int64_t)j * nf + r] : (r == j ? 1.0 : 0.0);
        };
        // backward coefficient of output i and row r: Linv(r, i), or -W(r, i)
        auto bwd_a = [&](int t, int r, int i) {
            const int nf = fs.nf[t], ns = fs.ns[t];
            if (r >= ns) return -front(t)[(int64_t)i * nf + r];
            return r > i ? front(t)[(int64_t)i * nf + r] : (r == i ? 1.0 : 0.0);
        };
        std::vector<double> acc(nrhs);
        // one front of the forward sweep: Y_s = Linv X_s, X_b -= W X_s (k_solve_fwd_inv)
        auto fwd_front = [&](int t) {
            const int nf = fs.nf[t], ns = fs.ns[t], ps = fs.pstart[t];
            for (int r = 0; r < nf; ++r) {
                std::fill(acc.begin(), acc.end(), 0.0);
                for (int j = 0; j < ns; ++j) {
                    const double a = fwd_a(t, r, j);
                    if (a != 0.0)
                        for (int c = 0; c < nrhs; ++c) acc[c] += a * Xi[(size_t)(ps + j) * nrhs + c];
                }
                if (r < ns) {
                    for (int c = 0; c < nrhs; ++c) Y[(size_t)(ps + r) * nrhs + c] = acc[c];
                } else {
                    const int g = row(t, r);
                    for (int c = 0; c < nrhs; ++c) Xi[(size_t)g * nrhs + c] -= acc[c];
                }
            }
        };
        // one front of the backward sweep: X_s = Linv^T D^-1 Y_s - W^T X_b (k_solve_bwd_inv)
        auto bwd_front = [&](int t) {
            const int nf = fs.nf[t], ns = fs.ns[t], ps = fs.pstart[t];
            for (int i = 0; i < ns; ++i) {
                std::fill(acc.begin(), acc.end(), 0.0);
                for (int r = i; r < nf; ++r) {
                    const double a = bwd_a(t, r, i);
                    if (r < ns) {
                        const double di = dinv(t, r);
                        for (int c = 0; c < nrhs; ++c) acc[c] += a * Y[(size_t)(ps + r) * nrhs + c] * di;
                    } else {
                        const int g = row(t, r);
                        for (int c = 0; c < nrhs; ++c) acc[c] += a * Xi[(size_t)g * nrhs + c];
                    }
                }
                for (int c = 0; c < nrhs; ++c) Xi[(size_t)(ps + i) * nrhs + c] = acc[c];
            }
        };
        // heights 0 and 1 fused as k_solve_fwd_fused / k_solve_bwd_fused order
        // them: a parent's rows held apart (pivot values and ancestor deltas),
        // D^-1 Y stored by the forward for these fronts
        k::FusePlan Fp;
        const bool fused = fused_h01 && fs.max_height >= 1;
        if (fused) Fp = k::fuse_plan(fs.nf, fs.ns, fs.parent, fs.by_height[0], fs.by_height[1], k::kFuseSmemCap);
        std::vector<double> Xp;
        auto fwd_fused = [&](int i) {
            const int pf = Fp.par[i], nfP = fs.nf[pf], nsP = fs.ns[pf], psP = fs.pstart[pf];
            Xp.assign((size_t)nfP * nrhs, 0.0);
            for (int r = 0; r < nsP; ++r)
                for (int c = 0; c < nrhs; ++c) Xp[(size_t)r * nrhs + c] = Xi[(size_t)(psP + r) * nrhs + c];
            for (int e = Fp.cptr[i]; e < Fp.cptr[i + 1]; ++e) {
                const int t = Fp.cid[e], nf = fs.nf[t], ns = fs.ns[t], ps = fs.pstart[t];
                const int *rel = fs.relmap.data() + fs.relmap_off[t];
                for (int r = 0; r < nf; ++r) {
                    std::fill(acc.begin(), acc.end(), 0.0);
                    for (int j = 0; j < ns; ++j) {
                        const double a = fwd_a(t, r, j);
                        for (int c = 0; c < nrhs; ++c) acc[c] += a * Xi[(size_t)(ps + j) * nrhs + c];
                    }
                    if (r < ns) {
                        const double di = dinv(t, r);
                        for (int c = 0; c < nrhs; ++c) Y[(size_t)(ps + r) * nrhs + c] = acc[c] * di;
                    } else {
                        const int pr = rel[r - ns];
                        if (pr < 0 || pr >= nfP) fail(HSIM_E_INTERNAL, "relmap outside the parent");
                        const double sg = pr < nsP ? -1.0 : 1.0;  // a pivot value, or a delta
                        for (int c = 0; c < nrhs; ++c) Xp[(size_t)pr * nrhs + c] += sg * acc[c];
                    }
                }
            }
            for (int r = 0; r < nfP; ++r) {
                std::fill(acc.begin(), acc.end(), 0.0);
                for (int j = 0; j < nsP; ++j) {
                    const double a = fwd_a(pf, r, j);
                    for (int c = 0; c < nrhs; ++c) acc[c] += a * Xp[(size_t)j * nrhs + c];
                }
                if (r < nsP) {
                    const double di = dinv(pf, r);
                    for (int c = 0; c < nrhs; ++c) Y[(size_t)(psP + r) * nrhs + c] = acc[c] * di;
                } else {
                    for (int c = 0; c < nrhs; ++c) Xp[(size_t)r * nrhs + c] += acc[c];
                }
            }
            for (int r = nsP; r < nfP; ++r) {
                const int g = row(pf, r);
                for (int c = 0; c < nrhs; ++c) Xi[(size_t)g * nrhs + c] -= Xp[(size_t)r * nrhs + c];
            }
        };
        auto bwd_fused = [&](int i) {
            const int pf = Fp.par[i], nfP = fs.nf[pf], nsP = fs.ns[pf], psP = fs.pstart[pf];
            Xp.assign((size_t)nfP * nrhs, 0.0);
            for (int r = 0; r < nfP; ++r) {
                const size_t src = r < nsP ? (size_t)(psP + r) : (size_t)row(pf, r);
                const double *from = r < nsP ? Y.data() : Xi.data();
                for (int c = 0; c < nrhs; ++c) Xp[(size_t)r * nrhs + c] = from[src * nrhs + c];
            }
            std::vector<double> out((size_t)nsP * nrhs, 0.0);
            for (int o = 0; o < nsP; ++o)
                for (int r = o; r < nfP; ++r) {
                    const double a = bwd_a(pf, r, o);
                    for (int c = 0; c < nrhs; ++c) out[(size_t)o * nrhs + c] += a * Xp[(size_t)r * nrhs + c];
                }
            for (int o = 0; o < nsP; ++o)
                for (int c = 0; c < nrhs; ++c) {
                    Xp[(size_t)o * nrhs + c] = out[(size_t)o * nrhs + c];
                    Xi[(size_t)(psP + o) * nrhs + c] = out[(size_t)o * nrhs + c];
                }
            for (int e = Fp.cptr[i]; e < Fp.cptr[i + 1]; ++e) {
                const int t = Fp.cid[e], nf = fs.nf[t], ns = fs.ns[t], ps = fs.pstart[t];
                const int *rel = fs.relmap.data() + fs.relmap_off[t];
                for (int o = 0; o < ns; ++o) {
                    std::fill(acc.begin(), acc.end(), 0.0);
                    for (int r = o; r < nf; ++r) {
                        const double a = bwd_a(t, r, o);
                        const double *b = r < ns ? &Y[(size_t)(ps + r) * nrhs] : &Xp[(size_t)rel[r - ns] * nrhs];
                        for (int c = 0; c < nrhs; ++c) acc[c] += a * b[c];
                    }
                    for (int c = 0; c < nrhs; ++c) Xi[(size_t)(ps + o) * nrhs + c] = acc[c];
                }
            }
        };
        for (int h = 0; h <= fs.max_height; ++h) {
            if (fused && h == 0) {
                for (int t : Fp.rest0) fwd_front(t);
                for (size_t i = 0; i < Fp.par.size(); ++i) fwd_fused((int)i);
            } else if (fused && h == 1) {
                for (int t : Fp.rest1) fwd_front(t);
            } else {
                for (int t : fs.by_height[h]) fwd_front(t);
            }
        }
        for (int h = fs.max_height; h >= 0; --h) {
            if (fused && h == 1) {
                for (int t : Fp.rest1) bwd_front(t);
                for (size_t i = 0; i < Fp.par.size(); ++i) bwd_fused((int)i);
            } else if (fused && h == 0) {
                for (int t : Fp.rest0) bwd_front(t);
            } else {
                for (int t : fs.by_height[h]) bwd_front(t);
            }
        }
        if (fused_counts) {
            fused_counts[0] = fused ? (int)Fp.par.size() : 0;
            fused_counts[1] = fused ? (int)Fp.rest0.size() : 0;
            fused_counts[2] = fused ? (int)Fp.rest1.size() : 0;
        }
        for (int pos = 0; pos < n; ++pos)
            std::memcpy(&X[(size_t)fs.perm[pos] * nrhs], &Xi[(size_t)pos * nrhs], nrhs * sizeof(double));
        if (neg_pivots) *neg_pivots = neg;
        if (nnz_L) *nnz_L = fs.nnz_L;
        return HSIM_OK;
    } catch (...) {
        return caught();
    }
}

extern "C" hsim_status hsim_check_hierarchy(int n, int m, const double *V, const int32_t *F, const double *L2, int p,
                                            const hsim_options *opts, int *levels, int *sizes, int64_t *U_nnz,
                                            int64_t *nnz0, int32_t *dofs, int32_t *order, int32_t *U_ptr,
                                            int32_t *U_col, double *U_val, int32_t *ptr0, int32_t *col0,
                                            int64_t *src0) {
    try {
        HSIM_CHECK_ARG(levels && sizes && U_nnz && nnz0, "NULL argument");
        hsim_options o;
        hsim_default_options(&o);
        if (opts) o = *opts;
        const int q = o.q > 0 ? o.q : std::max((int)std::ceil(1.5 * p), p + 8);
        HSIM_CHECK_ARG(o.boundary == HSIM_BOUNDARY_NATURAL || o.boundary == HSIM_BOUNDARY_DIRICHLET,
                       "unknown boundary condition");
        HSIM_CHECK_ARG(o.plain_sim == 0 || o.plain_sim == 1, "plain_sim must be 0 or 1");
        HostHierarchy h = build_host_hierarchy(n, m, V, F, L2, p, o.plain_sim ? 1 : o.levels, o.start_vertex, o.sigma,
                                               q, o.boundary == HSIM_BOUNDARY_DIRICHLET);
        const int T = (int)h.sizes.size();
        *levels = T;
        for (int t = 0; t < T; ++t) sizes[t] = h.sizes[t];
        for (int t = 0; t + 1 < T; ++t) U_nnz[t] = h.U[t].nnz();
        if (dofs)
            for (int i = 0; i < h.sizes[0]; ++i) dofs[i] = h.dofs.empty() ? i : h.dofs[i];
        // level-0 pattern and, per entry, the mesh entry (row * n + col) its value comes from
        *nnz0 = h.A0.nnz();
        if (ptr0) std::memcpy(ptr0, h.A0.ptr.data(), h.A0.ptr.size() * sizeof(int32_t));
        if (col0) std::memcpy(col0, h.A0.col.data(), h.A0.col.size() * sizeof(int32_t));
        if (src0) {
            std::vector<int> row_of(h.A_mesh.nnz());
            for (int i = 0; i < h.A_mesh.n_rows; ++i)
                for (int e = h.A_mesh.ptr[i]; e < h.A_mesh.ptr[i + 1]; ++e) row_of[e] = i;
            for (int64_t k = 0; k < h.A0.nnz(); ++k) {
                const int64_t e = h.smap.empty() ? k : h.smap[k];
                src0[k] = (int64_t)row_of[e] * n + h.A_mesh.col[e];
            }
        }
        if (order && !h.order.empty()) std::memcpy(order, h.order.data(), h.order.size() * sizeof(int32_t));
        int64_t po = 0, eo = 0;
        for (int t = 0; t + 1 < T; ++t) {
            const Csr &U = h.U[t];
            if (U_ptr) std::memcpy(U_ptr + po, U.ptr.data(), U.ptr.size() * sizeof(int32_t));
            if (U_col) std::memcpy(U_col + eo, U.col.data(), U.col.size() * sizeof(int32_t));
            if (U_val) std::memcpy(U_val + eo, U.val.data(), U.val.size() * sizeof(double));
            po += (int64_t)U.ptr.size();
            eo += U.nnz();
        }
        return HSIM_OK;
    } catch (...) {
        return caught();
    }
}

extern "C" hsim_status hsim_check_plain_basis(int n, const double *sdiag, const double *mdiag, const int32_t *perm,
                                              int q, uint64_t seed, int32_t *unit_pos, double *rand_int) {
    try {
        HSIM_CHECK_ARG(sdiag && mdiag && perm && unit_pos && rand_int, "NULL argument");
        std::vector<int> p(perm, perm + n), ip(n, -1);
        for (int i = 0; i < n; ++i) {
            HSIM_CHECK_ARG(p[i] >= 0 && p[i] < n && ip[p[i]] < 0, "perm is not a permutation");
            ip[p[i]] = i;
        }
        std::vector<int> up;
        std::vector<double> rc;
        plain_basis(n, sdiag, mdiag, p.data(), ip.data(), q, seed, &up, &rc);
        std::memcpy(unit_pos, up.data(), up.size() * sizeof(int32_t));
        std::memcpy(rand_int, rc.data(), rc.size() * sizeof(double));
        return HSIM_OK;
    } catch (...) {
        return caught();
    }
}
