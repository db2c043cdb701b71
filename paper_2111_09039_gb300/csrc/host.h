// Host-side structures: mesh graph, hierarchy construction and the symbolic
// analysis (nested dissection + supernodal fronts) of each level's matrix.
#pragma once

#include <cstdint>
#include <vector>

#include "common.h"

namespace hsim {

struct MeshGraph {
    int n = 0, m = 0;
    std::vector<int> ptr, idx;  // sorted neighbours
    std::vector<double> w;      // edge lengths
    std::vector<double> l2;     // per triangle, squared length opposite each corner
    double area = 0.0;
};

MeshGraph build_mesh_graph(int n, int m, const double *V, const int *F, const double *L2);
std::vector<int> level_sizes(int n, int p, int levels);
// Endpoints of the edges that exactly one triangle holds, ascending.
std::vector<int> boundary_vertices(int n, int m, const int *F);
// Farthest-point order (Alg. 2); with cand, only vertices with cand[v] != 0
// are chosen (distances still run over the whole graph).
std::vector<int> farthest_point_order(const MeshGraph &g, int start, int count,
                                      const std::vector<char> *cand = nullptr);
// U^tau; for fine_is_mesh the rows are the mesh vertices, or the vertices
// listed in dofs (ascending) when dofs is given.
Csr prolongation(const MeshGraph &g, const std::vector<int> &order, int nf, int nc,
                 bool fine_is_mesh, double sigma, double *rho_out, int *fallback_rows,
                 const std::vector<int> *dofs = nullptr);

// The mesh-dependent part of a hierarchy (Sec. 4.1): level sizes, the
// farthest-point order of Alg. 2 and every prolongation U^tau in natural
// (mesh / sampling) order.  levels <= 0 selects 3, or 2 when p <= 200; the
// subspace size q must fit the coarsest level.  With a Dirichlet boundary
// the boundary vertices are eliminated and the construction runs over the
// interior vertices: level sizes from their count, sampling among them only,
// U^0 rows for the interior vertices in increasing id.
struct HostHierarchy {
    MeshGraph g;
    std::vector<int> dofs;      // Dirichlet: interior vertex ids (empty: every vertex)
    Csr A_mesh;                 // every mesh edge plus the diagonal (assembly pattern)
    Csr A0;                     // level-0 pattern: A_mesh, or its interior rows and columns
    std::vector<int64_t> smap;  // Dirichlet: entry of A_mesh behind each entry of A0
    std::vector<int> sizes;     // n^tau, tau = 0..T-1 (at most 8 levels)
    std::vector<int> order;     // first n^1 vertices of farthest-point sampling
    std::vector<Csr> U;         // U^tau: n^tau x n^{tau+1}, tau = 0..T-2
    std::vector<double> rho;    // support radius of U^tau
    std::vector<int> fallback;  // rows of U^tau with no centre inside rho
};
HostHierarchy build_host_hierarchy(int n, int m, const double *V, const int *F, const double *L2, int p,
                                   int levels, int start_vertex, double sigma, int q, bool dirichlet);
// The two halves of build_host_hierarchy: the mesh graph, the degrees of
// freedom, the level-0 patterns and the level sizes; then the sampling order
// and the prolongations (the long sequential part, which the caller may
// overlap with the symbolic analysis of A0).
HostHierarchy host_levels(int n, int m, const double *V, const int *F, const double *L2, int p, int levels,
                          int start_vertex, double sigma, int q, bool dirichlet);
void host_samples(HostHierarchy &h, int start_vertex, double sigma);
// The same sampling order and prolongations computed on the current CUDA
// device (k_hier.cu), equal index for index and bit for bit; V (host, n x 3)
// lets farthest-point sampling take several samples per relaxation (NULL for
// meshes given by edge lengths).
void device_samples(HostHierarchy &h, const double *V, int start_vertex, double sigma, cudaStream_t s);

namespace k {
// edge graph (and coordinates) of the mesh on the device
struct DeviceGraph {
    int n = 0, n_sm = 1, max_degree = 0;
    double area = 0.0;
    DevBuf<int> ptr, idx;
    DevBuf<double> w, V;
    void upload(const MeshGraph &g, const double *V_host, cudaStream_t s);
};
std::vector<int> fps_device(cudaStream_t s, const DeviceGraph &g, int start, int count,
                            const std::vector<char> *cand);
Csr prolongation_device(cudaStream_t s, const DeviceGraph &g, const std::vector<int> &order, int nf, int nc,
                        bool fine_is_mesh, double sigma, double *rho_out, int *fallback_rows,
                        const std::vector<int> *dofs);
}  // namespace k

// out[i] = 2 u_i - 1, u_i = (i-th SplitMix64 output from state seed) >> 11
// times 2^-53: the random column of plain SIM's initial basis.
void random_column(int n, uint64_t seed, double *out);

// Host part of plain SIM's initial basis (Sec. 3.2, initialisation
// heuristic) for a level whose elimination order is perm (perm[pos] =
// natural index, iperm its inverse): unit_pos[c] = internal row of the unit
// vector of column 1 + c (the q - 2 smallest sdiag/mdiag, ascending, the
// lower natural index first on ties); rand_int[pos] = random_column(seed) at
// natural index perm[pos].
void plain_basis(int n, const double *sdiag, const double *mdiag, const int *perm, const int *iperm, int q,
                 uint64_t seed, std::vector<int> *unit_pos, std::vector<double> *rand_int);

// ---- sparse pattern algebra -------------------------------------------
Csr mesh_pattern(const MeshGraph &g);                 // edges + diagonal, sorted
Csr transpose_pattern(const Csr &A);                  // pattern (and values if present)
Csr pattern_product(const Csr &A, const Csr &B);      // pattern of A*B (sorted)
Csr permute_symmetric(const Csr &A, const std::vector<int> &iperm,
                      std::vector<int64_t> *value_map);  // P A P^T, map new entry -> old entry
Csr permute_rows_cols(const Csr &A, const std::vector<int> &row_iperm,
                      const std::vector<int> &col_iperm);  // with values
// A restricted to the rows and columns in keep (ascending), renumbered
// 0..|keep|-1; value_map: new entry -> entry of A.
Csr restrict_pattern(const Csr &A, const std::vector<int> &keep, std::vector<int64_t> *value_map);

// ---- supernodal symbolic analysis ---------------------------------------
// Fronts are the nodes of a nested-dissection tree: every leaf domain and
// every separator is one dense front (a supernode).  Positions are indices
// in the internal (elimination) order.
struct FrontSymbolic {
    int n = 0;
    std::vector<int> perm;   // perm[pos] = natural index
    std::vector<int> iperm;  // iperm[natural] = pos
    int n_nodes = 0;
    std::vector<int> pstart, ns, nf, parent, height, nsteps;
    std::vector<int64_t> rows_off;   // node -> offset into rows (nf entries)
    std::vector<int> rows;           // front row lists (positions), pivots first
    std::vector<int64_t> foff;       // node -> arena offset (column-major nf x nf)
    int64_t arena = 0;
    std::vector<int64_t> relmap_off; // node -> offset into relmap (nf - ns entries)
    std::vector<int> relmap;         // struct row -> parent-local row
    int max_height = 0;
    // per height: nodes sorted by decreasing panel-step count
    std::vector<std::vector<int>> by_height;
    // per height: children (of nodes at this height) that feed an extend-add
    std::vector<std::vector<int>> ea_children;
    std::vector<int> pos_node;       // pos -> owning node
    int64_t nnz_L = 0;
    double flops = 0.0;
    int max_front = 0;
};

constexpr int kPanel = 32;  // panel width of the blocked front kernels

// Nested dissection of the symmetric pattern A (natural order, diagonal
// ignored) and the front structure of the permuted matrix.
FrontSymbolic analyse(const Csr &A, int leaf_size);

// Destination offsets in the front arena of every entry of the
// internal-order CSR A (already permuted by fs.perm) in the lower triangle
// (-1 for upper entries).
std::vector<int64_t> assembly_map(const FrontSymbolic &fs, const Csr &A_internal);

}  // namespace hsim
