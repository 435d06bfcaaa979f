// The paper's naive path (Section III), kept as the comparator of the batched
// kernels: RVEs are solved one after another; each iteration of Algorithm 1 is
// a short sequence of launches over one RVE (a fused free-DOF update, a
// zeroing kernel and an atomic scatter for getInternalForces, a fused
// damping/acceleration/velocity kernel with the residual reduction) and the
// host reads the residual back every iteration to test convergence.
// Plain FP64 with the compiler's default contraction; the atomic scatter makes
// the summation order, and hence the chaotic trajectory, run-dependent.
#include <algorithm>
#include <cmath>

#include "dr_device.cuh"

namespace fe2 {
namespace naive {

__global__ void k_affine(int n, const double *X0, const double *X1, const double *X2,
                         const double *F, double *x0, double *x1, double *x2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = X0[i], b = X1[i], c = X2[i];
    x0[i] = F[0] * a + F[1] * b + F[2] * c;
    x1[i] = F[3] * a + F[4] * b + F[5] * c;
    x2[i] = F[6] * a + F[7] * b + F[8] * c;
}

__global__ void k_init(int n, int nf, int init, const double *X0, const double *X1,
                       const double *X2, double *x0, double *x1, double *x2, double *u0,
                       double *u1, double *u2, double *v0, double *v1, double *v2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool fixed = i >= nf;
    double ua[3] = {x0[i] - X0[i], x1[i] - X1[i], x2[i] - X2[i]};
    double u[3];
    for (int r = 0; r < 3; ++r) {
        if (fixed || init == 1) u[r] = ua[r];
        else if (init == 2) u[r] = r == 0 ? u0[i] : (r == 1 ? u1[i] : u2[i]);
        else u[r] = 0.0;
    }
    u0[i] = u[0]; u1[i] = u[1]; u2[i] = u[2];
    x0[i] = X0[i] + u[0]; x1[i] = X1[i] + u[1]; x2[i] = X2[i] + u[2];
    if (!fixed) { v0[i] = 0.0; v1[i] = 0.0; v2[i] = 0.0; }
}

__global__ void k_zero(int n3, double *g) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) g[i] = 0.0;
}

// getInternalForces, second kernel: element forces scattered with atomics.
__global__ void k_scatter(int ne, const int32_t *ea, const int32_t *eb, const double *EA,
                          const double *L, const double *x0, const double *x1, const double *x2,
                          double *g0, double *g1, double *g2) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    const int a = ea[e], b = eb[e];
    const double d0 = x0[b] - x0[a], d1 = x1[b] - x1[a], d2 = x2[b] - x2[a];
    const double l = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const double q = EA[e] * (l / L[e] - 1.0) / l;
    atomicAdd(g0 + a, q * d0); atomicAdd(g1 + a, q * d1); atomicAdd(g2 + a, q * d2);
    atomicAdd(g0 + b, -q * d0); atomicAdd(g1 + b, -q * d1); atomicAdd(g2 + b, -q * d2);
}

__device__ __forceinline__ void reduce_add(double v, double *out) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(out, t);
    }
}

__global__ void k_norm_accel0(int n, int nf, const double *m, const double *g0, const double *g1,
                              const double *g2, double *a0, double *a1, double *a2, double *acc,
                              int set_accel) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < n) {
        s = g0[i] * g0[i] + g1[i] * g1[i] + g2[i] * g2[i];
        if (set_accel && i < nf) { a0[i] = g0[i] / m[i]; a1[i] = g1[i] / m[i]; a2[i] = g2[i] / m[i]; }
    }
    reduce_add(s, acc);
}

// Partial velocity update and displacement update (free DOFs, fused).
__global__ void k_half_disp(int nf, double hdt, double dt, const double *X0, const double *X1,
                            const double *X2, const double *a0, const double *a1, const double *a2,
                            double *v0, double *v1, double *v2, double *u0, double *u1, double *u2,
                            double *x0, double *x1, double *x2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    v0[i] += hdt * a0[i]; v1[i] += hdt * a1[i]; v2[i] += hdt * a2[i];
    u0[i] += dt * v0[i]; u1[i] += dt * v1[i]; u2[i] += dt * v2[i];
    x0[i] = X0[i] + u0[i]; x1[i] = X1[i] + u1[i]; x2[i] = X2[i] + u2[i];
}

// Damping force, residual (reduction), accelerations, partial velocity update.
__global__ void k_accel(int nf, double mc, double hdt, const double *m, const double *g0,
                        const double *g1, const double *g2, double *v0, double *v1, double *v2,
                        double *a0, double *a1, double *a2, double *acc) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (i < nf) {
        const double mi = m[i];
        const double g[3] = {g0[i], g1[i], g2[i]};
        double *v[3] = {v0 + i, v1 + i, v2 + i};
        double *a[3] = {a0 + i, a1 + i, a2 + i};
        for (int r = 0; r < 3; ++r) {
            const double fd = mc * mi * *v[r];
            s += g[r] * g[r];
            *a[r] = (g[r] + fd) / mi;
            *v[r] += hdt * *a[r];
        }
    }
    reduce_add(s, acc);
}

__global__ void k_stress(int ne, const int32_t *ea, const int32_t *eb, const double *EA,
                         const double *L, const double *x0, const double *x1, const double *x2,
                         double *acc9) {
    __shared__ double red[9][32];
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (e < ne) {
        const int a = ea[e], b = eb[e];
        const double d[3] = {x0[b] - x0[a], x1[b] - x1[a], x2[b] - x2[a]};
        const double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double q = EA[e] * (l / L[e] - 1.0) / l;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) s[3 * r + c] = q * d[r] * d[c];
    }
    for (int k = 0; k < 9; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
        atomicAdd(acc9 + threadIdx.x, t);
    }
}

__global__ void k_finish(const double *acc9, const double *F, double V0, double *sigma) {
    if (threadIdx.x < 9) sigma[threadIdx.x] = acc9[threadIdx.x] / (det3(F) * V0);
}

}  // namespace naive

// One RVE through the naive loop. Returns 0 or a cudaError_t.
int naive_solve_rve(const RveDesc &R, const DevMesh &M, const DevState &S, const DevResults &O,
                    const double *F_dev, const NaiveScratch &W, double tol, int64_t max_iter,
                    double alpha, int init, int p, cudaStream_t st, int64_t *iters_out,
                    double *rel_out, int *status_out) {
    using namespace naive;
    const int n = R.n_nodes, nf = R.n_free, ne = R.n_elems;
    const int64_t n0 = R.node0;
    const int T = 256;
    const int gn = (n + T - 1) / T, gf = (nf + T - 1) / T > 0 ? (nf + T - 1) / T : 1,
              ge = (ne + T - 1) / T > 0 ? (ne + T - 1) / T : 1, g3 = (3 * n + T - 1) / T;
    double *x0 = W.x, *x1 = W.x + n, *x2 = W.x + 2 * n;
    double *g0 = W.g, *g1 = W.g + n, *g2 = W.g + 2 * n;
    const double *X0 = M.X0 + n0, *X1 = M.X1 + n0, *X2 = M.X2 + n0;
    double *u0 = S.u0 + n0, *u1 = S.u1 + n0, *u2 = S.u2 + n0;
    double *v0 = S.v0 + n0, *v1 = S.v1 + n0, *v2 = S.v2 + n0;
    double *a0 = S.a0 + n0, *a1 = S.a1 + n0, *a2 = S.a2 + n0;
    const double *m = M.mass + n0;
    const int32_t *ea = M.el_a + R.elem0, *eb = M.el_b + R.elem0;
    const double *EA = M.el_EA + R.elem0, *L = M.el_L + R.elem0;
    const double *F = F_dev + 9 * (int64_t)p;
    double h[2];
    cudaError_t e;
#define NV_CHECK() do { e = cudaGetLastError(); if (e != cudaSuccess) return (int)e; } while (0)
    // f_ref: |g(F X)| over all DOFs
    k_affine<<<gn, T, 0, st>>>(n, X0, X1, X2, F, x0, x1, x2);
    k_zero<<<g3, T, 0, st>>>(3 * n, W.g);
    if (ne) k_scatter<<<ge, T, 0, st>>>(ne, ea, eb, EA, L, x0, x1, x2, g0, g1, g2);
    cudaMemsetAsync(W.acc, 0, 3 * sizeof(double), st);
    k_norm_accel0<<<gn, T, 0, st>>>(n, nf, m, g0, g1, g2, a0, a1, a2, W.acc, 0);
    // initial state, forces and accelerations
    k_init<<<gn, T, 0, st>>>(n, nf, init, X0, X1, X2, x0, x1, x2, u0, u1, u2, v0, v1, v2);
    k_zero<<<g3, T, 0, st>>>(3 * n, W.g);
    if (ne) k_scatter<<<ge, T, 0, st>>>(ne, ea, eb, EA, L, x0, x1, x2, g0, g1, g2);
    k_norm_accel0<<<gn, T, 0, st>>>(n, nf, m, g0, g1, g2, a0, a1, a2, W.acc + 1, 1);
    NV_CHECK();
    e = cudaMemcpyAsync(h, W.acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return (int)e;
    const double f_ref = std::max(std::sqrt(h[0]), std::sqrt(h[1]));
    const double dt = alpha * R.dtc, hdt = 0.5 * dt, mc = -R.c;
    int64_t it = 0;
    int status = RVE_MAXITER;
    double r = 0.0;
    for (;;) {
        k_half_disp<<<gf, T, 0, st>>>(nf, hdt, dt, X0, X1, X2, a0, a1, a2, v0, v1, v2, u0, u1, u2,
                                      x0, x1, x2);
        k_zero<<<g3, T, 0, st>>>(3 * n, W.g);
        if (ne) k_scatter<<<ge, T, 0, st>>>(ne, ea, eb, EA, L, x0, x1, x2, g0, g1, g2);
        k_accel<<<gf, T, 0, st>>>(nf, mc, hdt, m, g0, g1, g2, v0, v1, v2, a0, a1, a2, W.acc + 2);
        NV_CHECK();
        // residual to the host every iteration (a blocking reduction)
        e = cudaMemcpyAsync(h, W.acc + 2, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(W.acc + 2, 0, sizeof(double), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return (int)e;
        r = std::sqrt(h[0]);
        ++it;
        if (!std::isfinite(r)) { status = RVE_NAN; break; }
        if (r <= tol * f_ref) { status = RVE_OK; break; }
        if (it >= max_iter) { status = RVE_MAXITER; break; }
    }
    cudaMemsetAsync(W.acc + 4, 0, 9 * sizeof(double), st);
    if (ne) k_stress<<<ge, T, 0, st>>>(ne, ea, eb, EA, L, x0, x1, x2, W.acc + 4);
    k_finish<<<1, 32, 0, st>>>(W.acc + 4, F, R.V0, O.sigma + 9 * (int64_t)p);
    NV_CHECK();
    *iters_out = it;
    *rel_out = f_ref > 0.0 ? r / f_ref : (r > 0.0 ? INFINITY : 0.0);
    *status_out = status;
    return 0;
#undef NV_CHECK
}

}  // namespace fe2
