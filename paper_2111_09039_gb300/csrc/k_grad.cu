// Shape gradient of a loss of the eigenvalues (first-order perturbation of
// S Phi = lambda M Phi for M-normalised eigenvectors, applied to the cotan
// stiffness and lumped mass of Sec. 3.1):
//
//     dL/dx_v = sum_i w_i phi_i^T (dS/dx_v - lambda_i dM/dx_v) phi_i,
//     w_i = dL/dlambda_i.
//
// Per triangle with corners x_0, x_1, x_2 the quadratic forms are
//     phi^T S phi |_t = 1/2 sum_k cot_k (phi_{k+1} - phi_{k+2})^2,
//     phi^T M phi |_t = A_t / 3 sum_k phi_k^2,
// so one pass over the eigenpairs reduces every triangle to four numbers,
//     D_k = sum_i w_i (phi_i(k+1) - phi_i(k+2))^2,  P = sum_i w_i lambda_i sum_k phi_i(k)^2,
// and the gradient is 1/2 sum_k D_k dcot_k/dx - P/3 dA/dx.  Here the corner
// cotangent is written with the two edge vectors leaving the corner,
// u = x_{k+1} - x_k, w = x_{k+2} - x_k, cot_k = (u.w) / |u x w|, and with
// n = (u x w)/|u x w| (the same for all three corners),
//     d cot_k = [ (w - cot_k (w x n)) . du + (u - cot_k (n x u)) . dw ] / |u x w|,
//     d A     = 1/2 [ (w x n) . du + (n x u) . dw ]         (corner 0).
// One thread per triangle; the nine partial derivatives go to the vertices
// with FP64 atomics (the order of the additions, hence the last bits, vary
// from run to run).

#include "common.h"
#include "kernels.h"

namespace hsim {
namespace k {

namespace {

struct v3 {
    double x, y, z;
};
__device__ __forceinline__ v3 sub(v3 a, v3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ v3 add(v3 a, v3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ v3 mul(double s, v3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ v3 cross(v3 a, v3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ v3 load(const double *V, int v) {
    return {V[3 * (size_t)v], V[3 * (size_t)v + 1], V[3 * (size_t)v + 2]};
}
__device__ __forceinline__ void atomic_add3(double *g, int v, v3 a) {
    atomicAdd(g + 3 * (size_t)v, a.x);
    atomicAdd(g + 3 * (size_t)v + 1, a.y);
    atomicAdd(g + 3 * (size_t)v + 2, a.z);
}

__global__ void __launch_bounds__(256) k_eig_grad(int m, int n, int p, const double *__restrict__ V,
                                                  const int *__restrict__ F, const double *__restrict__ evals,
                                                  const double *__restrict__ evecs, int ld,
                                                  const double *__restrict__ dl, double *__restrict__ g) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    int c[3] = {F[3 * (size_t)t], F[3 * (size_t)t + 1], F[3 * (size_t)t + 2]};
    double D[3] = {0.0, 0.0, 0.0}, P = 0.0;
    for (int i = 0; i < p; ++i) {
        double w = __ldg(dl + i);
        if (w == 0.0) continue;
        const double *phi = evecs + (size_t)i * ld;
        double f0 = __ldg(phi + c[0]), f1 = __ldg(phi + c[1]), f2 = __ldg(phi + c[2]);
        double d0 = f1 - f2, d1 = f2 - f0, d2 = f0 - f1;
        D[0] += w * d0 * d0;
        D[1] += w * d1 * d1;
        D[2] += w * d2 * d2;
        P += w * __ldg(evals + i) * (f0 * f0 + f1 * f1 + f2 * f2);
    }
    v3 x[3] = {load(V, c[0]), load(V, c[1]), load(V, c[2])};
    v3 nrm = cross(sub(x[1], x[0]), sub(x[2], x[0]));
    double s = sqrt(dot(nrm, nrm));  // 2 A
    nrm = mul(1.0 / s, nrm);
    v3 gr[3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int k = 0; k < 3; ++k) {
        int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        v3 u = sub(x[k1], x[k]), w = sub(x[k2], x[k]);
        double cot = dot(u, w) / s;
        double h = 0.5 * D[k] / s;
        v3 gu = mul(h, sub(w, mul(cot, cross(w, nrm))));
        v3 gw = mul(h, sub(u, mul(cot, cross(nrm, u))));
        gr[k1] = add(gr[k1], gu);
        gr[k2] = add(gr[k2], gw);
        gr[k] = sub(gr[k], add(gu, gw));
    }
    // - P/3 dA/dx
    double a = -P / 6.0;
    v3 ga1 = mul(a, cross(sub(x[2], x[0]), nrm));
    v3 ga2 = mul(a, cross(nrm, sub(x[1], x[0])));
    gr[1] = add(gr[1], ga1);
    gr[2] = add(gr[2], ga2);
    gr[0] = sub(gr[0], add(ga1, ga2));
    for (int k = 0; k < 3; ++k) atomic_add3(g, c[k], gr[k]);
}

}  // namespace

void eig_grad(cudaStream_t s, int n, int m, int p, const double *V, const int *F, const double *evals,
              const double *evecs, int ld, const double *dloss, double *dV) {
    HSIM_CUDA(cudaMemsetAsync(dV, 0, sizeof(double) * 3 * (size_t)n, s));
    if (m == 0) return;
    k_eig_grad<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, n, p, V, F, evals, evecs, ld, dloss, dV);
    HSIM_LAUNCHED();
}

}  // namespace k
}  // namespace hsim
