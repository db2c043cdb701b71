// Vertex hierarchy on the GPU (Sec. 4.1): farthest-point sampling (Alg. 2)
// and the prolongation operators U^tau (eqs. radius and basis), with the
// same results, index for index and bit for bit, as the host construction.
//
// Distances.  Every distance is the least rounded path sum over the edge
// graph (the rounded sum is monotone in its first operand, so any order of
// relaxations that ends with no improving edge reaches it): the searches
// here are frontier-based Bellman-Ford rounds with an atomic minimum on the
// bit pattern of the non-negative FP64 distance, and they reach the values of
// the host's bucket queue and of a textbook Dijkstra exactly.
//
// Farthest-point sampling.  Sample k + 1 is the vertex of largest distance to
// samples 0..k (ties to the lowest id).  One CTA keeps the distance field's
// per-block maxima (blocks of kB consecutive vertices) in a tournament tree
// in shared memory.  The chain of 3 * 10^4 dependent choices is shortened by
// taking several samples per relaxation: after the field's maximum c1 is
// taken, the next candidate c2 (the next largest value) is also the next
// sample if c1's distance update cannot lower it, which holds when the
// straight-line distance |x_c1 - x_c2| is at least dist(c2): the graph's
// edge weights are the edges' Euclidean lengths, so a path is never shorter
// than the straight line (with a relative margin of 10^-6 for rounding).
// Candidates are taken in order while each passes this test against every
// sample already in the batch; the batch is then relaxed from all its members
// at once (the minimum over sources does not depend on the order).  Meshes
// given by intrinsic edge lengths have no coordinates and take one sample per
// relaxation.
//
// Prolongations.  One truncated search per centre (distance < rho), centres
// spread over CTAs that each own a distance array over the whole mesh; the
// entries (row, centre, 1 - d / rho) are counted per row, scattered, sorted
// by centre within each row and normalised by their sum in centre order.  A
// row with no centre inside the radius takes weight one on its nearest centre
// (multi-source search; ties to the lowest centre index, found by
// propagating the least centre index along the edges on shortest paths).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <mutex>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "common.h"
#include "host.h"
#include "kernels.h"

namespace hsim {
namespace k {

namespace cg = cooperative_groups;

namespace {

constexpr int kFpsThreads = 1024;
constexpr int kFpsWarps = kFpsThreads / 32;
constexpr int kFpsBatch = 256;       // samples per relaxation at most
constexpr int kFpsSlots = 8;         // threads per frontier vertex (one per edge slot)
constexpr int kFpsMaxCluster = 16;   // CTAs of the sampling cluster at most
constexpr int kFpsSoloItems = 2048;  // frontier items (vertex x slot) that CTA 0 relaxes alone
constexpr int kFpsSoloQueue = 2048;  // frontier entries of the solo rounds kept in shared memory
constexpr int kFpsMaxLeaves = 4096;  // tournament-tree leaves (shared memory)
constexpr int kFpsMaxBlock = 2048;   // vertices per block at most (meshes up to 2^23 vertices)
constexpr double kFpsMargin = 1e-6;  // relative margin of the straight-line test
constexpr double kFpsMarginSq = (1.0 - kFpsMargin) * (1.0 - kFpsMargin);
constexpr int kBallThreads = 256;
// dynamic shared memory of k_fps for L leaves: the tree's distances and
// vertices, the batch's coordinates and vertices
constexpr size_t fps_smem(int L) { return 2 * (size_t)L * 12 + 3 * kFpsBatch * 8 + kFpsBatch * 4; }
constexpr size_t kFpsMaxSmem = fps_smem(kFpsMaxLeaves);
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// lower *d to nd if nd is smaller; true if this call lowered it (d >= 0 and
// nd >= 0, so the bit patterns order like the values)
__device__ __forceinline__ bool lower(double *d, double nd, unsigned long long *old_out = nullptr) {
    const unsigned long long nb = (unsigned long long)__double_as_longlong(nd);
    const unsigned long long old = atomicMin(reinterpret_cast<unsigned long long *>(d), nb);
    if (old_out) *old_out = old;
    return nb < old;
}

__global__ void k_fill_f64(int64_t n, double v, double *x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}
__global__ void k_fill_i32(int64_t n, int v, int *x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

void fill(cudaStream_t s, int64_t n, double v, double *x) {
    if (n <= 0) return;
    k_fill_f64<<<std::min<int64_t>(cdiv(n, 256), 4096), 256, 0, s>>>(n, v, x);
    HSIM_LAUNCHED();
}
void fill(cudaStream_t s, int64_t n, int v, int *x) {
    if (n <= 0) return;
    k_fill_i32<<<std::min<int64_t>(cdiv(n, 256), 4096), 256, 0, s>>>(n, v, x);
    HSIM_LAUNCHED();
}

// ---- farthest-point sampling ----------------------------------------------------

struct FpsArgs {
    int n;
    const int *ptr, *idx;
    const double *w;
    const double *V;             // n x 3 coordinates, or null (one sample per relaxation)
    const unsigned char *cand;   // candidates (null: every vertex)
    int start, count, kB, nb, L;
    double *dist;                // n, +inf on entry
    int *stamp;                  // n, -1 on entry
    int *q;                      // 2 buffers x C segments x n: frontier queues, one segment per CTA
    unsigned *dbm;               // nb bits: block's maximum out of date (all set on entry)
    int *dirty;                  // nb: the flagged blocks, listed after each relaxation
    int *dirty_cnt;              // 0 on entry
    int *order;                  // count
    int *status;                 // [0]: 0, 1 relaxation did not settle, 2 no candidate left; [1]: done
    int solo_dup;                // solo rounds may push a vertex twice (see relax_items)
};

// Tournament tree over the blocks: node i holds the farthest candidate of its
// subtree, (distance td[i], vertex tv[i]; tv = -1: none); leaves L + b.
// Node i takes the farther of its children (larger distance, the lower vertex
// on ties).
__device__ __forceinline__ void tree_update(double *td, int *tv, int i) {
    const double d0 = td[2 * i], d1 = td[2 * i + 1];
    const int v0 = tv[2 * i], v1 = tv[2 * i + 1];
    const bool left = v0 >= 0 && (v1 < 0 || d0 > d1 || (d0 == d1 && v0 < v1));
    td[i] = left ? d0 : d1;
    tv[i] = left ? v0 : v1;
}

// (bd, best) = the farther of (bd, best) and (od, ob)
__device__ __forceinline__ void farther(double &bd, int &best, double od, int ob) {
    if (ob >= 0 && (best < 0 || od > bd || (od == bd && ob < best))) {
        best = ob;
        bd = od;
    }
}
__device__ __forceinline__ void warp_farthest(double &bd, int &best) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const int ob = __shfl_xor_sync(0xffffffffu, best, o);
        const double od = __shfl_xor_sync(0xffffffffu, bd, o);
        farther(bd, best, od, ob);
    }
}

// The farthest candidate of block b, by one warp, skipping the block
// positions whose bit is set in skip (null: none): (bd, best) in every lane,
// best = -1 if none.  The lanes read 8 vertices each per 256-vertex chunk,
// all loads first.
__device__ __forceinline__ void block_max(const FpsArgs &a, int b, int lane, const unsigned *skip, double &bd,
                                          int &best) {
    best = -1;
    bd = -1.0;
    const int v0 = b * a.kB, v1 = min(a.n, v0 + a.kB);
    for (int c0 = v0; c0 < v1; c0 += 256) {
        constexpr int R = 8;
        double d[R];
        bool in[R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int v = c0 + lane + 32 * t;
            in[t] = v < v1 && (!a.cand || a.cand[v]);
            if (in[t] && skip) in[t] = !((skip[(v - v0) >> 5] >> ((v - v0) & 31)) & 1u);
            d[t] = in[t] ? __ldcg(a.dist + v) : 0.0;
        }
#pragma unroll
        for (int t = 0; t < R; ++t) {
            const int v = c0 + lane + 32 * t;
            if (in[t] && (best < 0 || d[t] > bd)) {  // ascending v per lane: ties keep the lower id
                best = v;
                bd = d[t];
            }
        }
    }
    warp_farthest(bd, best);
}

// block_max written to leaf b of (td, tv) by lane 0
__device__ __forceinline__ void rescan_block(const FpsArgs &a, int b, double *td, int *tv, int lane) {
    double bd;
    int best;
    block_max(a, b, lane, nullptr, bd, best);
    if (lane == 0) {
        td[b] = bd;
        tv[b] = best;
    }
}

// flag block b as out of date (no result: the relaxation does not wait for it)
__device__ __forceinline__ void mark_dirty(const FpsArgs &a, int b) { atomicOr(a.dbm + (b >> 5), 1u << (b & 31)); }

// One Bellman-Ford round r over the frontier (the first nseg segments of queue
// buffer r & 1 with cnt[k] entries each): items it = first, first + stride,
// ... of (frontier vertex, edge slot); a neighbour whose distance drops is
// pushed once into this CTA's segment `rank` of buffer (r + 1) & 1 and its
// block flagged.
// SOLO (CTA 0 alone, at most kFpsSoloItems items): the atomic minimum is
// issued without a plain load first, and with a.solo_dup a neighbour lowered
// twice in the round is pushed twice (the host allows it when a round's
// pushes, at most kFpsSoloItems / kFpsSlots vertices times the largest
// degree, fit in a segment); a duplicate is expanded twice with the same
// distance, which changes nothing.
//
// sq_in / sq_out (solo rounds, shared memory): the first kFpsSoloQueue
// entries of segment 0 of the current / next frontier are read from / pushed
// to shared memory instead of the global queue (later entries stay global).
template <bool SOLO>
__device__ __forceinline__ void relax_items(const FpsArgs &a, int r, const int *cnt, int nseg, int64_t first,
                                            int64_t stride, size_t qbuf, int rank, int *s_cnt, const int *sq_in,
                                            int *sq_out) {
    const int *qc = a.q + (size_t)(r & 1) * qbuf;
    int *qn = a.q + (size_t)((r + 1) & 1) * qbuf + (size_t)rank * a.n;
    const int tag = r + 1;
    int total = 0;
    for (int k = 0; k < nseg; ++k) total += cnt[k];
    const int64_t items = (int64_t)total * kFpsSlots;
    for (int64_t it = first; it < items; it += stride) {
        int j = (int)(it / kFpsSlots);
        const int slot = (int)(it % kFpsSlots);
        int seg = 0;
        while (j >= cnt[seg]) j -= cnt[seg++];
        const int v = (sq_in && seg == 0 && j < kFpsSoloQueue) ? sq_in[j] : qc[(size_t)seg * a.n + j];
        const int e0 = a.ptr[v], e1 = a.ptr[v + 1];
        const double dv = __ldcg(a.dist + v);
        for (int e = e0 + slot; e < e1; e += kFpsSlots) {
            const int u = a.idx[e];
            const double nd = dv + a.w[e];
            if ((SOLO || nd < __ldcg(a.dist + u)) && lower(a.dist + u, nd)) {
                if ((SOLO && a.solo_dup) || atomicExch(a.stamp + u, tag) != tag) {
                    const int pos = atomicAdd(&s_cnt[(r + 1) % 3], 1);
                    if (sq_out && pos < kFpsSoloQueue) sq_out[pos] = u;
                    else qn[pos] = u;
                }
                mark_dirty(a, u / a.kB);
            }
        }
    }
}

// One cluster of C CTAs.  CTA 0 holds the tournament tree and forms the
// batches; all CTAs relax the frontier (one queue segment per CTA, the
// frontier of a round being the concatenation of the segments) and rescan
// the changed blocks, writing the blocks' maxima into CTA 0's shared memory.
// Rounds are separated by the cluster barrier.
__global__ void __launch_bounds__(kFpsThreads, 1) k_fps(const FpsArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), C = (int)cl.num_blocks();
    extern __shared__ __align__(16) unsigned char sm[];
    const int L = a.L;
    double *td = reinterpret_cast<double *>(sm);                  // 2L tree distances
    double *bx = td + 2 * L;                                      // kFpsBatch x 3
    int *tv = reinterpret_cast<int *>(bx + 3 * kFpsBatch);        // 2L tree vertices
    int *bv = tv + 2 * L;                                         // kFpsBatch
    __shared__ int s_cnt[3];  // pushes into this CTA's segment, by round mod 3
    __shared__ int s_nbatch, s_norder, s_r;
    __shared__ long long s_rounds;
    __shared__ unsigned s_skip[kFpsMaxBlock / 32];  // batch members in the block being rescanned
    __shared__ int s_q[2][kFpsSoloQueue];          // frontier queues of the solo rounds
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    double *leafd0 = cl.map_shared_rank(td, 0) + L;
    int *leafv0 = cl.map_shared_rank(tv, 0) + L;

    if (rank == 0)
        for (int i = tid; i < 2 * L; i += kFpsThreads) {
            td[i] = -1.0;
            tv[i] = -1;
        }
    if (tid == 0) {
        s_cnt[0] = s_cnt[1] = s_cnt[2] = 0;
        s_nbatch = 1;
        s_norder = 0;
        bv[0] = a.start;
    }
    cl.sync();
    int r = 0;  // round index, the same in every thread of the cluster
    const size_t qbuf = (size_t)C * a.n;
    for (;;) {
        // CTA 0 inserts the batch: distance zero, frontier of round r
        if (rank == 0) {
            const int nbt = s_nbatch, no = s_norder;
            int *q0 = a.q + (size_t)(r & 1) * qbuf;
            for (int j = tid; j < nbt; j += kFpsThreads) {
                const int sv = bv[j];
                a.order[no + j] = sv;
                lower(a.dist + sv, 0.0);
                q0[j] = sv;
                mark_dirty(a, sv / a.kB);
            }
            __syncthreads();
            if (tid == 0) {
                s_cnt[r % 3] = nbt;
                s_norder = no + nbt;
            }
        }
        cl.sync();
        // Bellman-Ford rounds following improving edges only.  While the
        // frontier is small, CTA 0 runs the rounds alone (block barriers
        // instead of cluster barriers) and hands a larger frontier back.
        int64_t rounds = 0;
        for (;;) {
            int cnt[kFpsMaxCluster];
            int total = 0;
            for (int k = 0; k < C; ++k) {
                cnt[k] = *cl.map_shared_rank(&s_cnt[r % 3], k);
                total += cnt[k];
            }
            if (total == 0) break;
            if (C > 1 && (int64_t)total * kFpsSlots <= kFpsSoloItems) {
                if (rank == 0) {
                    int nseg = C, tot = 0;
                    bool in_smem = false;  // the frontier's first entries are in s_q[r & 1]
                    for (;;) {
                        tot = 0;
                        for (int k = 0; k < nseg; ++k) tot += cnt[k];
                        if (tot == 0 || (int64_t)tot * kFpsSlots > kFpsSoloItems) break;
                        if (++rounds > (int64_t)a.n + 2) {
                            if (tid == 0) atomicExch(a.status, 1);
                            break;
                        }
                        if (tid == 0) s_cnt[(r + 2) % 3] = 0;
                        relax_items<true>(a, r, cnt, nseg, tid, kFpsThreads, qbuf, 0, s_cnt,
                                          in_smem ? s_q[r & 1] : nullptr, s_q[(r + 1) & 1]);
                        in_smem = true;
                        ++r;
                        __syncthreads();
                        cnt[0] = s_cnt[r % 3];  // pushes of this CTA only from now on
                        nseg = 1;
                    }
                    // a frontier handed back to the cluster goes to the global queue
                    if (in_smem && tot > 0) {
                        int *qg = a.q + (size_t)(r & 1) * qbuf;
                        for (int j = tid; j < min(tot, kFpsSoloQueue); j += kFpsThreads) qg[j] = s_q[r & 1][j];
                    }
                    if (tid == 0) {
                        s_r = r;
                        s_rounds = rounds;
                    }
                    // the whole frontier is in this CTA's segment: clear the others' counts
                    for (int k = 1 + tid; k < C; k += kFpsThreads) {
                        int *o = cl.map_shared_rank(s_cnt, k);
                        o[0] = o[1] = o[2] = 0;
                    }
                }
                cl.sync();
                r = *cl.map_shared_rank(&s_r, 0);
                rounds = *cl.map_shared_rank(&s_rounds, 0);
                if (__ldcg(a.status) != 0) return;  // uniform after the barrier
                continue;
            }
            if (++rounds > (int64_t)a.n + 2) {  // uniform: every thread counts the same rounds
                if (rank == 0 && tid == 0) atomicExch(a.status, 1);
                return;
            }
            if (tid == 0) s_cnt[(r + 2) % 3] = 0;  // read by everyone in round r - 1
            relax_items<false>(a, r, cnt, C, (int64_t)rank * kFpsThreads + tid, (int64_t)C * kFpsThreads, qbuf, rank,
                               s_cnt, nullptr, nullptr);
            ++r;
            cl.sync();
        }
        // list the flagged blocks (all CTAs over the flag words)
        const int nwords = (a.nb + 31) >> 5;
        for (int wd = rank * kFpsThreads + tid; wd < nwords; wd += C * kFpsThreads) {
            unsigned bits = __ldcg(a.dbm + wd);
            if (!bits) continue;
            __stcg(a.dbm + wd, 0u);
            const int pos = atomicAdd(a.dirty_cnt, __popc(bits));
            for (int k = 0; bits; ++k) {
                const int b = (wd << 5) + __ffs(bits) - 1;
                bits &= bits - 1;
                a.dirty[pos + k] = b;
            }
        }
        cl.sync();
        // rescan the blocks whose distances changed (all CTAs), then CTA 0
        // updates their tree paths and forms the next batch
        const int ndirty = __ldcg(a.dirty_cnt);
        for (int k = rank * kFpsWarps + warp; k < ndirty; k += C * kFpsWarps) {
            const int b = a.dirty[k];
            rescan_block(a, b, leafd0, leafv0, lane);
        }
        cl.sync();
        if (rank == 0) {
            for (int lvl = 1; (L >> lvl) >= 1; ++lvl) {
                for (int k = tid; k < ndirty; k += kFpsThreads) tree_update(td, tv, (L + a.dirty[k]) >> lvl);
                __syncthreads();
            }
            if (tid == 0) atomicExch(a.dirty_cnt, 0);
            if (s_norder >= a.count) {
                if (tid == 0) atomicExch(a.status + 1, 1);
            } else if (warp == 0) {
                // candidates in order while each is farther, in a straight
                // line, from every member than its own distance; a taken
                // candidate's block is rescanned without the batch's members
                int nb = 0;
                const int norder = s_norder;
                for (;;) {
                    const int c = tv[1];
                    if (c < 0) break;
                    const double dc = td[1];
                    const int b = c / a.kB, v0 = b * a.kB;
                    // c's block without c and the batch's members, computed
                    // before the test so that its loads overlap c's coordinates
                    for (int i = lane; i < (a.kB >> 5); i += 32) s_skip[i] = 0u;
                    __syncwarp();
                    if (lane == 0) atomicOr(&s_skip[(c - v0) >> 5], 1u << ((c - v0) & 31));
                    for (int j = lane; j < nb; j += 32) {
                        const int m = bv[j] - v0;
                        if (m >= 0 && m < a.kB) atomicOr(&s_skip[m >> 5], 1u << (m & 31));
                    }
                    __syncwarp();
                    double cx = 0.0, cy = 0.0, cz = 0.0;
                    if (a.V) {
                        cx = a.V[3 * (int64_t)c];
                        cy = a.V[3 * (int64_t)c + 1];
                        cz = a.V[3 * (int64_t)c + 2];
                    }
                    double bd;
                    int best;
                    block_max(a, b, lane, s_skip, bd, best);
                    if (nb > 0) {
                        bool ok = a.V != nullptr && dc > 0.0;
                        if (ok)
                            for (int j = lane; j < nb; j += 32) {
                                // |x_j - x_c| (1 - margin) >= dc, compared squared
                                const double dx = bx[3 * j] - cx, dy = bx[3 * j + 1] - cy, dz = bx[3 * j + 2] - cz;
                                const double e2 = dx * dx + dy * dy + dz * dz;
                                if (!(e2 * kFpsMarginSq >= dc * dc)) ok = false;
                            }
                        if (!__all_sync(0xffffffffu, ok)) break;
                    }
                    if (lane == 0) {
                        bv[nb] = c;
                        bx[3 * nb] = cx;
                        bx[3 * nb + 1] = cy;
                        bx[3 * nb + 2] = cz;
                        td[L + b] = bd;
                        tv[L + b] = best;
                        for (int i = (L + b) >> 1; i >= 1; i >>= 1) tree_update(td, tv, i);
                    }
                    ++nb;
                    __syncwarp();
                    if (norder + nb >= a.count || nb >= kFpsBatch) break;
                }
                if (lane == 0) {
                    s_nbatch = nb;
                    if (nb == 0) atomicExch(a.status, 2);
                }
            }
        }
        cl.sync();
        if (__ldcg(a.status) != 0 || __ldcg(a.status + 1) != 0) return;  // uniform after the barrier
    }
}

// ---- truncated searches of the prolongations -------------------------------------

struct BallArgs {
    int n;
    const int *ptr, *idx;
    const double *w;
    const int *centre;   // mesh vertex of centre c (c < nc)
    int nc;
    double rho;
    const int *rowmap;   // fine row of a mesh vertex or -1 (null: the vertex id itself)
    int nf;
    double *dist;        // gridDim.x x n, +inf on entry (left so on exit)
    int *stamp;          // gridDim.x x n, -1 on entry
    int *qa, *qb, *touched;  // gridDim.x x n each
    int *row_count;      // nf
    unsigned long long *cursor;  // entries written (may exceed cap: then nothing past cap is stored)
    int64_t cap;
    int *ent_row, *ent_col;
    double *ent_w;
    int *status;
};

__global__ void __launch_bounds__(kBallThreads) k_balls(const BallArgs a) {
    __shared__ int s_nfront, s_nnext, s_ntouched;
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * a.n;
    double *dist = a.dist + base;
    int *stamp = a.stamp + base, *qa = a.qa + base, *qb = a.qb + base, *touched = a.touched + base;
    int rid = 0;
    for (int c = blockIdx.x; c < a.nc; c += gridDim.x) {
        const int sv = a.centre[c];
        if (tid == 0) {
            dist[sv] = 0.0;
            qa[0] = sv;
            touched[0] = sv;
            s_nfront = 1;
            s_nnext = 0;
            s_ntouched = 1;
        }
        __syncthreads();
        int *qc = qa, *qn = qb;
        int64_t rounds = 0;
        for (;;) {
            const int nfr = s_nfront;
            if (nfr == 0) break;
            if (++rounds > (int64_t)a.n + 2) {
                if (tid == 0) atomicExch(a.status, 1);
                break;
            }
            ++rid;
            for (int i = tid; i < nfr; i += kBallThreads) {
                const int v = qc[i];
                const double dv = __ldcg(dist + v);
                for (int e = a.ptr[v]; e < a.ptr[v + 1]; ++e) {
                    const int u = a.idx[e];
                    const double nd = dv + a.w[e];
                    unsigned long long old;
                    if (nd < a.rho && nd < __ldcg(dist + u) && lower(dist + u, nd, &old)) {
                        if (old == kInfBits) touched[atomicAdd(&s_ntouched, 1)] = u;
                        if (atomicExch(stamp + u, rid) != rid) qn[atomicAdd(&s_nnext, 1)] = u;
                    }
                }
            }
            __syncthreads();
            if (tid == 0) {
                s_nfront = s_nnext;
                s_nnext = 0;
            }
            int *t = qc;
            qc = qn;
            qn = t;
            __syncthreads();
        }
        const int nt = s_ntouched;
        for (int i = tid; i < nt; i += kBallThreads) {
            const int v = touched[i];
            const double d = __ldcg(dist + v);
            const int row = a.rowmap ? a.rowmap[v] : v;
            if (row >= 0 && row < a.nf) {
                atomicAdd(a.row_count + row, 1);
                const unsigned long long k = atomicAdd(a.cursor, 1ull);
                if ((int64_t)k < a.cap) {
                    a.ent_row[k] = row;
                    a.ent_col[k] = c;
                    a.ent_w[k] = 1.0 - d / a.rho;
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < nt; i += kBallThreads) dist[touched[i]] = INFINITY;
        __syncthreads();
    }
}

// ---- nearest centre of the rows without a centre inside the radius ---------------

__global__ void k_ms_relax(int nfr, const int *__restrict__ front, const int *__restrict__ ptr,
                           const int *__restrict__ idx, const double *__restrict__ w, double *nd, int *stamp, int rid,
                           int *next, int *nnext) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nfr; i += gridDim.x * blockDim.x) {
        const int v = front[i];
        const double dv = __ldcg(nd + v);
        for (int e = ptr[v]; e < ptr[v + 1]; ++e) {
            const int u = idx[e];
            const double d = dv + w[e];
            if (d < __ldcg(nd + u) && lower(nd + u, d))
                if (atomicExch(stamp + u, rid) != rid) next[atomicAdd(nnext, 1)] = u;
        }
    }
}

// label[u] = least label over the neighbours v on a shortest path to u
// (nd[v] + w == nd[u]); *changed set when a label decreased
__global__ void k_label_round(int n, const int *__restrict__ ptr, const int *__restrict__ idx,
                              const double *__restrict__ w, const double *__restrict__ nd, int *label, int *changed) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const double du = nd[u];
        int best = __ldcg(label + u);
        for (int e = ptr[u]; e < ptr[u + 1]; ++e) {
            const int v = idx[e];
            if (nd[v] + w[e] == du) best = min(best, __ldcg(label + v));
        }
        if (best < __ldcg(label + u)) {
            atomicMin(label + u, best);
            *changed = 1;
        }
    }
}

__global__ void k_centre_labels(int nc, const int *__restrict__ centre, double *nd, int *label, int *front) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
        nd[centre[c]] = 0.0;
        atomicMin(label + centre[c], c);
        front[c] = centre[c];
    }
}

// ---- rows of U -----------------------------------------------------------------

// fallback entries of the rows with no entry; *missing counts them, *bad a
// row whose vertex no centre reaches
__global__ void k_fallback_rows(int nf, int *row_count, const int *__restrict__ fine_vertex, const int *__restrict__ label,
                                unsigned long long *cursor, int64_t cap, int *ent_row, int *ent_col, double *ent_w,
                                int *missing, int *bad) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nf; r += gridDim.x * blockDim.x) {
        if (row_count[r] != 0) continue;
        atomicAdd(missing, 1);
        if (!label) continue;
        const int v = fine_vertex ? fine_vertex[r] : r;
        const int c = label[v];
        if (c == INT_MAX) {
            atomicExch(bad, 1);
            continue;
        }
        row_count[r] = 1;
        const unsigned long long k = atomicAdd(cursor, 1ull);
        if ((int64_t)k < cap) {
            ent_row[k] = r;
            ent_col[k] = c;
            ent_w[k] = 1.0;
        }
    }
}

// exclusive prefix sum of count[0..n) into ptr[0..n], one CTA of 1024 threads
__global__ void __launch_bounds__(1024) k_scan_counts(int n, const int *__restrict__ count, int *ptr) {
    __shared__ int part[1024];
    const int tid = threadIdx.x;
    const int chunk = (n + 1023) / 1024;
    const int b = min(n, tid * chunk), e = min(n, b + chunk);
    int s = 0;
    for (int i = b; i < e; ++i) s += count[i];
    part[tid] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int v = tid >= o ? part[tid - o] : 0;
        __syncthreads();
        part[tid] += v;
        __syncthreads();
    }
    int run = tid > 0 ? part[tid - 1] : 0;
    for (int i = b; i < e; ++i) {
        ptr[i] = run;
        run += count[i];
    }
    if (tid == 1023) ptr[n] = part[1023];
}

__global__ void k_scatter_entries(int64_t ne, const int *__restrict__ ent_row, const int *__restrict__ ent_col,
                                  const double *__restrict__ ent_w, const int *__restrict__ ptr, int *fillc, int *col,
                                  double *val) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ne; k += (int64_t)gridDim.x * blockDim.x) {
        const int r = ent_row[k];
        const int pos = ptr[r] + atomicAdd(fillc + r, 1);
        col[pos] = ent_col[k];
        val[pos] = ent_w[k];
    }
}

// sort each row by centre index, then divide by the row sum taken in that order
__global__ void k_sort_normalise(int nf, const int *__restrict__ ptr, int *col, double *val) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nf; r += gridDim.x * blockDim.x) {
        const int b = ptr[r], e = ptr[r + 1];
        for (int i = b + 1; i < e; ++i) {
            const int c = col[i];
            const double v = val[i];
            int j = i - 1;
            while (j >= b && col[j] > c) {
                col[j + 1] = col[j];
                val[j + 1] = val[j];
                --j;
            }
            col[j + 1] = c;
            val[j + 1] = v;
        }
        double sum = 0.0;
        for (int i = b; i < e; ++i) sum += val[i];
        for (int i = b; i < e; ++i) val[i] /= sum;
    }
}

__global__ void k_rank_rows(int nf, const int *__restrict__ order, int *rowmap) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nf; k += gridDim.x * blockDim.x) rowmap[order[k]] = k;
}

int read_int(cudaStream_t s, const int *p) {
    int h = 0;
    HSIM_CUDA(cudaMemcpyAsync(&h, p, sizeof(int), cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaStreamSynchronize(s));
    return h;
}

}  // namespace

void DeviceGraph::upload(const MeshGraph &g, const double *V_host, cudaStream_t s) {
    n = g.n;
    area = g.area;
    max_degree = 0;
    for (int v = 0; v < g.n; ++v) max_degree = std::max(max_degree, g.ptr[v + 1] - g.ptr[v]);
    ptr.upload(g.ptr, s);
    idx.upload(g.idx, s);
    w.upload(g.w, s);
    if (V_host) {
        V.alloc(3 * (size_t)g.n);
        HSIM_CUDA(cudaMemcpyAsync(V.p, V_host, 3 * (size_t)g.n * sizeof(double), cudaMemcpyHostToDevice, s));
    } else {
        V.release();
    }
    int sms = 0, dev = 0;
    HSIM_CUDA(cudaGetDevice(&dev));
    HSIM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    n_sm = std::max(1, sms);
}

std::vector<int> fps_device(cudaStream_t s, const DeviceGraph &g, int start, int count, const std::vector<char> *cand) {
    const int n = g.n;
    HSIM_CHECK_ARG(start >= 0 && start < n, "start vertex out of range");
    HSIM_CHECK_ARG(!cand || (*cand)[start], "start vertex is not a degree of freedom");
    int ncand = n;
    if (cand) ncand = (int)std::count_if(cand->begin(), cand->end(), [](char c) { return c != 0; });
    HSIM_CHECK_ARG(count >= 1 && count <= ncand, "bad sample count");
    // blocks of kB vertices (a multiple of 32), at most kFpsMaxLeaves blocks
    const int kB = 32 * std::max(1, (int)cdiv(n, 32LL * kFpsMaxLeaves));
    HSIM_CHECK_ARG(kB <= kFpsMaxBlock, "mesh too large for the GPU farthest-point sampling (2^23 vertices at most)");
    const int nb = (int)cdiv(n, kB);
    int L = 1;
    while (L < nb) L *= 2;
    const size_t smem = fps_smem(L);
    HSIM_SMEM_LIMIT_ONCE(k_fps, kFpsMaxSmem);
    static std::once_flag np_once;
    std::call_once(np_once, [] { cudaFuncSetAttribute(k_fps, cudaFuncAttributeNonPortableClusterSizeAllowed, 1); });
    cudaGetLastError();
    // the largest cluster (16, else 8, 4, 2, 1 CTAs) that can be resident
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.blockDim = dim3(kFpsThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    int C = kFpsMaxCluster;
    for (; C > 1; C /= 2) {
        cfg.gridDim = dim3(C);
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        int active = 0;
        if (cudaOccupancyMaxActiveClusters(&active, k_fps, &cfg) == cudaSuccess && active >= 1) break;
        cudaGetLastError();
    }
    cfg.gridDim = dim3(C);
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    DevBuf<double> dist(n);
    DevBuf<int> stamp(n), q(2 * (size_t)C * n), dirty(nb), order(count), status(2), dirty_cnt(1);
    DevBuf<unsigned> dbm(cdiv(nb, 32));
    DevBuf<unsigned char> dcand;
    if (cand) {
        std::vector<unsigned char> c8(cand->begin(), cand->end());
        dcand.alloc(n);
        HSIM_CUDA(cudaMemcpyAsync(dcand.p, c8.data(), n, cudaMemcpyHostToDevice, s));
        HSIM_CUDA(cudaStreamSynchronize(s));  // c8 leaves scope
    }
    fill(s, n, INFINITY, dist.p);
    fill(s, n, -1, stamp.p);
    fill(s, 2, 0, status.p);
    fill(s, 1, 0, dirty_cnt.p);
    // every block out of date (bits past nb stay clear)
    std::vector<unsigned> bits(cdiv(nb, 32), 0xffffffffu);
    if (nb % 32) bits.back() = (1u << (nb % 32)) - 1u;
    HSIM_CUDA(cudaMemcpyAsync(dbm.p, bits.data(), bits.size() * sizeof(unsigned), cudaMemcpyHostToDevice, s));
    // a solo round pushes at most (kFpsSoloItems / kFpsSlots) * max_degree entries
    const int solo_dup = (int64_t)(kFpsSoloItems / kFpsSlots) * g.max_degree <= n ? 1 : 0;
    FpsArgs a{n, g.ptr.p, g.idx.p, g.w.p, g.V.p, dcand.p, start, count, kB, nb, L, dist.p, stamp.p, q.p,
              dbm.p, dirty.p, dirty_cnt.p, order.p, status.p, solo_dup};
    HSIM_CUDA(cudaLaunchKernelEx(&cfg, k_fps, a));
    HSIM_LAUNCHED();
    const int st = read_int(s, status.p);
    if (st == 1) fail(HSIM_E_INTERNAL, "farthest-point sampling: a distance relaxation did not settle");
    if (st == 2) fail(HSIM_E_INTERNAL, "farthest-point sampling: no candidate left");
    return order.download(s);
}

Csr prolongation_device(cudaStream_t s, const DeviceGraph &g, const std::vector<int> &order, int nf, int nc,
                        bool fine_is_mesh, double sigma, double *rho_out, int *fallback_rows,
                        const std::vector<int> *dofs) {
    const int n = g.n;
    const double rho = std::sqrt(sigma * g.area / ((double)nc * M_PI));
    *rho_out = rho;
    HSIM_CHECK_ARG(nc >= 1 && nc <= (int)order.size(), "bad centre count");
    DevBuf<int> dorder;
    dorder.upload(order, s);
    // fine row of every mesh vertex, and mesh vertex of every fine row
    DevBuf<int> rowmap, fine_vertex;
    if (fine_is_mesh && dofs) {
        std::vector<int> row_of(n, -1);
        for (int k = 0; k < (int)dofs->size(); ++k) row_of[(*dofs)[k]] = k;
        rowmap.upload(row_of, s);
        fine_vertex.upload(*dofs, s);
    } else if (!fine_is_mesh) {
        rowmap.alloc(n);
        fill(s, n, -1, rowmap.p);
        k_rank_rows<<<cdiv(nf, 256), 256, 0, s>>>(nf, dorder.p, rowmap.p);
        HSIM_LAUNCHED();
    }
    const int *fine_vertex_p = fine_is_mesh ? fine_vertex.p : dorder.p;  // null: row r is vertex r
    // one CTA per SM (each owns four arrays over the mesh), at most one per centre
    const int grid = std::max(1, std::min(nc, g.n_sm));
    DevBuf<double> dist((size_t)grid * n);
    DevBuf<int> stamp((size_t)grid * n), qa((size_t)grid * n), qb((size_t)grid * n), touched((size_t)grid * n);
    DevBuf<int> row_count(nf), status(2);
    DevBuf<unsigned long long> cursor(1);
    fill(s, (int64_t)grid * n, INFINITY, dist.p);
    int64_t cap = 8 * (int64_t)nf + 1024;  // about sigma entries per row expected
    DevBuf<int> ent_row, ent_col;
    DevBuf<double> ent_w;
    for (int attempt = 0;; ++attempt) {
        ent_row.alloc(cap);
        ent_col.alloc(cap);
        ent_w.alloc(cap);
        fill(s, (int64_t)grid * n, -1, stamp.p);  // round ids restart with every launch
        fill(s, nf, 0, row_count.p);
        fill(s, 2, 0, status.p);
        HSIM_CUDA(cudaMemsetAsync(cursor.p, 0, sizeof(unsigned long long), s));
        BallArgs a{n, g.ptr.p, g.idx.p, g.w.p, dorder.p, nc, rho, rowmap.p, nf, dist.p, stamp.p, qa.p, qb.p,
                   touched.p, row_count.p, cursor.p, cap, ent_row.p, ent_col.p, ent_w.p, status.p};
        k_balls<<<grid, kBallThreads, 0, s>>>(a);
        HSIM_LAUNCHED();
        unsigned long long ne = 0;
        HSIM_CUDA(cudaMemcpyAsync(&ne, cursor.p, sizeof(ne), cudaMemcpyDeviceToHost, s));
        HSIM_CUDA(cudaStreamSynchronize(s));
        if (read_int(s, status.p) != 0) fail(HSIM_E_INTERNAL, "prolongation: a truncated search did not settle");
        // room for the entries plus one fallback entry per row
        if ((int64_t)ne + nf <= cap) break;
        HSIM_CHECK_ARG(attempt == 0, "prolongation: entry count changed between runs");
        cap = (int64_t)ne + nf + 1024;
    }
    dist.release();
    stamp.release();
    touched.release();
    // rows without a centre inside the radius
    DevBuf<int> missing(2);
    fill(s, 2, 0, missing.p);
    k_fallback_rows<<<cdiv(nf, 256), 256, 0, s>>>(nf, row_count.p, nullptr, nullptr, cursor.p, cap, ent_row.p,
                                                  ent_col.p, ent_w.p, missing.p, missing.p + 1);
    HSIM_LAUNCHED();
    const int n_missing = read_int(s, missing.p);
    *fallback_rows = n_missing;
    if (n_missing > 0) {
        DevBuf<double> nd(n);
        DevBuf<int> label(n), st(n), cnt(1);
        fill(s, n, INFINITY, nd.p);
        fill(s, n, INT_MAX, label.p);
        fill(s, n, -1, st.p);
        k_centre_labels<<<cdiv(nc, 256), 256, 0, s>>>(nc, dorder.p, nd.p, label.p, qa.p);
        HSIM_LAUNCHED();
        int nfr = nc, rid = 0;
        int *qc = qa.p, *qn = qb.p;
        // a vertex whose distance stopped changing leaves the frontier; at
        // most n rounds with positive edge weights
        while (nfr > 0) {
            HSIM_CHECK_ARG(rid <= n + 2, "nearest-centre search did not settle");
            fill(s, 1, 0, cnt.p);
            k_ms_relax<<<std::min(cdiv(nfr, 256), 4096u), 256, 0, s>>>(nfr, qc, g.ptr.p, g.idx.p, g.w.p, nd.p, st.p,
                                                                       ++rid, qn, cnt.p);
            HSIM_LAUNCHED();
            nfr = read_int(s, cnt.p);
            std::swap(qc, qn);
        }
        for (int it = 0;; ++it) {
            HSIM_CHECK_ARG(it <= n + 2, "nearest-centre labels did not settle");
            fill(s, 1, 0, cnt.p);
            k_label_round<<<std::min(cdiv(n, 256), 4096u), 256, 0, s>>>(n, g.ptr.p, g.idx.p, g.w.p, nd.p, label.p,
                                                                       cnt.p);
            HSIM_LAUNCHED();
            if (read_int(s, cnt.p) == 0) break;
        }
        fill(s, 2, 0, missing.p);
        k_fallback_rows<<<cdiv(nf, 256), 256, 0, s>>>(nf, row_count.p, fine_vertex_p, label.p, cursor.p, cap,
                                                      ent_row.p, ent_col.p, ent_w.p, missing.p, missing.p + 1);
        HSIM_LAUNCHED();
        if (read_int(s, missing.p + 1) != 0)
            fail(HSIM_E_INVALID_ARG, "a connected component of the mesh holds no coarse vertex");
    }
    unsigned long long ne = 0;
    HSIM_CUDA(cudaMemcpyAsync(&ne, cursor.p, sizeof(ne), cudaMemcpyDeviceToHost, s));
    HSIM_CUDA(cudaStreamSynchronize(s));
    DevBuf<int> dptr(nf + 1), fillc(nf), dcol(std::max<int64_t>(1, (int64_t)ne));
    DevBuf<double> dval(std::max<int64_t>(1, (int64_t)ne));
    k_scan_counts<<<1, 1024, 0, s>>>(nf, row_count.p, dptr.p);
    HSIM_LAUNCHED();
    fill(s, nf, 0, fillc.p);
    HSIM_CHECK_ARG(ne >= (unsigned long long)nf, "prolongation: a row without entries");
    k_scatter_entries<<<std::min(cdiv((int64_t)ne, 256), 8192u), 256, 0, s>>>((int64_t)ne, ent_row.p, ent_col.p,
                                                                                 ent_w.p, dptr.p, fillc.p, dcol.p,
                                                                                 dval.p);
    HSIM_LAUNCHED();
    k_sort_normalise<<<cdiv(nf, 128), 128, 0, s>>>(nf, dptr.p, dcol.p, dval.p);
    HSIM_LAUNCHED();
    Csr U;
    U.n_rows = nf;
    U.n_cols = nc;
    U.ptr = dptr.download(s);
    U.col = dcol.download(s);
    U.val = dval.download(s);
    U.col.resize((size_t)ne);
    U.val.resize((size_t)ne);
    HSIM_CHECK_ARG(U.ptr[nf] == (int)ne, "prolongation: row counts disagree with the entries");
    return U;
}

}  // namespace k

void device_samples(HostHierarchy &h, const double *V, int start_vertex, double sigma, cudaStream_t s) {
    const int T = (int)h.sizes.size();
    const bool dirichlet = !h.dofs.empty();
    std::vector<char> interior;
    if (dirichlet) {
        interior.assign(h.g.n, 0);
        for (int v : h.dofs) interior[v] = 1;
    }
    // HSIM_TRACE set: wall time of each part on stderr
    const char *tr = std::getenv("HSIM_TRACE");
    const bool trace = tr && *tr && std::atoi(tr) > 0;
    auto t0 = std::chrono::steady_clock::now();
    auto lap = [&](const char *what) {
        if (!trace) return;
        HSIM_CUDA(cudaStreamSynchronize(s));
        const auto t1 = std::chrono::steady_clock::now();
        std::fprintf(stderr, "[hsim] device hierarchy: %s %.1f ms\n", what,
                     std::chrono::duration<double, std::milli>(t1 - t0).count());
        t0 = t1;
    };
    k::DeviceGraph dg;
    dg.upload(h.g, V, s);
    lap("graph upload");
    if (T > 1) h.order = k::fps_device(s, dg, start_vertex, h.sizes[1], dirichlet ? &interior : nullptr);
    lap("farthest-point sampling");
    h.U.resize(T - 1);
    h.rho.assign(T - 1, 0.0);
    h.fallback.assign(T - 1, 0);
    for (int tau = 0; tau + 1 < T; ++tau) {
        h.U[tau] = k::prolongation_device(s, dg, h.order, h.sizes[tau], h.sizes[tau + 1], tau == 0, sigma,
                                          &h.rho[tau], &h.fallback[tau], dirichlet ? &h.dofs : nullptr);
        lap(tau == 0 ? "prolongation U^0" : "prolongation U^tau (tau > 0)");
    }
}

}  // namespace hsim
