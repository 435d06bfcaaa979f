// Device helpers shared by the dynamic-relaxation kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fe2_internal.h"

namespace fe2 {

// ----------------------------------------------------------------------------
// IEEE FP64 with every rounding explicit (no FMA contraction): these are the
// operations, in the order, of a serial element-scatter implementation of
// Algorithm 1, so the trajectory matches one bit for bit.
// ----------------------------------------------------------------------------
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dsqrt(double a) { return __dsqrt_rn(a); }

// Sum over the CTA; every thread gets the total. `red` holds >= 32 doubles and
// must not be in use by another reduction until the next barrier.
__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = (blockDim.x + 31) >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    __syncthreads();
    return t;
}

__device__ __forceinline__ double det3(const double *F) {
    return dadd(dsub(dmul(F[0], dsub(dmul(F[4], F[8]), dmul(F[5], F[7]))),
                     dmul(F[1], dsub(dmul(F[3], F[8]), dmul(F[5], F[6])))),
                dmul(F[2], dsub(dmul(F[3], F[7]), dmul(F[4], F[6]))));
}

// Internal force on local node i (Algorithm 1, getInternalForces) as a gather
// over its CSR row: g_i = sum_j (N/l) (x_j - x_i), N = EA (l/L - 1), rows in
// ascending original neighbour id, so the partial sums equal those of the
// serial scatter (node a adds (N/l) d, node b subtracts it, d = x_b - x_a).
__device__ __forceinline__ void gather_force_fp64(const DevMesh &M, const int32_t *rowptr,
                                                  int64_t csr0, int i, const double *x0,
                                                  const double *x1, const double *x2,
                                                  double &g0, double &g1, double &g2) {
    const int beg = rowptr[i], end = rowptr[i + 1];
    const double xi0 = x0[i], xi1 = x1[i], xi2 = x2[i];
    g0 = 0.0; g1 = 0.0; g2 = 0.0;
    for (int k = beg; k < end; ++k) {
        const int64_t kk = csr0 + k;
        const int j = M.col[kk];
        const double d0 = dsub(x0[j], xi0), d1 = dsub(x1[j], xi1), d2 = dsub(x2[j], xi2);
        const double l = dsqrt(dadd(dadd(dmul(d0, d0), dmul(d1, d1)), dmul(d2, d2)));
        const double N = dmul(M.EA[kk], dsub(ddiv(l, M.L[kk]), 1.0));
        const double q = ddiv(N, l);
        g0 = dadd(g0, dmul(q, d0));
        g1 = dadd(g1, dmul(q, d1));
        g2 = dadd(g2, dmul(q, d2));
    }
}

// Volume-averaged Cauchy stress sigma = (1/V) sum_e (N_e/l_e) d_e (x) d_e over
// the RVE's elements, V = det(F) V0; thread 0 writes the 9 components.
__device__ inline void rve_stress(const DevMesh &M, const RveDesc &R, const double *F,
                                  const double *x0, const double *x1, const double *x2,
                                  double *sigma_out, double *red) {
    double s[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) s[k] = 0.0;
    for (int e = threadIdx.x; e < R.n_elems; e += blockDim.x) {
        const int64_t ee = R.elem0 + e;
        const int a = M.el_a[ee], b = M.el_b[ee];
        double d[3] = {dsub(x0[b], x0[a]), dsub(x1[b], x1[a]), dsub(x2[b], x2[a])};
        const double l = dsqrt(dadd(dadd(dmul(d[0], d[0]), dmul(d[1], d[1])), dmul(d[2], d[2])));
        const double q = ddiv(dmul(M.el_EA[ee], dsub(ddiv(l, M.el_L[ee]), 1.0)), l);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) s[3 * r + c] = dadd(s[3 * r + c], dmul(dmul(q, d[r]), d[c]));
    }
    const double V = dmul(det3(F), R.V0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const double t = block_sum(s[k], red);
        if (threadIdx.x == 0) sigma_out[k] = ddiv(t, V);
    }
}

}  // namespace fe2
