// FP64 oracle-order solve of one RVE by one CTA (Algorithm 1), shared by the
// persistent batch kernel and the allocation-free single-RVE entry point.
#pragma once
#include "dr_device.cuh"

namespace fe2 {

template <bool SM>
__device__ void solve_rve_fp64(const DevMesh &M, const DevState &S, const DevResults &O,
                               const SolveParams &P, int p, double *smem, double *red) {
    const RveDesc R = M.rve[p];
    const int n = R.n_nodes, nf = R.n_free;
    const int64_t n0 = R.node0;
    const int32_t *rowptr = M.rowptr + R.rp0;
    double *x0, *x1, *x2;
    if (SM) {
        x0 = smem;
    } else {
        x0 = S.xg + 3 * n0;
    }
    x1 = x0 + n;
    x2 = x1 + n;
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = P.F[9 * (int64_t)p + k];
    const double *X0 = M.X0 + n0, *X1 = M.X1 + n0, *X2 = M.X2 + n0;
    double *u0 = S.u0 + n0, *u1 = S.u1 + n0, *u2 = S.u2 + n0;
    double *v0 = S.v0 + n0, *v1 = S.v1 + n0, *v2 = S.v2 + n0;
    double *a0 = S.a0 + n0, *a1 = S.a1 + n0, *a2 = S.a2 + n0;
    const double *mass = M.mass + n0;

    // f_ref, part 1: forces in the affine configuration x = F X (all DOFs).
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double X[3] = {X0[i], X1[i], X2[i]};
        x0[i] = dadd(dadd(dmul(F[0], X[0]), dmul(F[1], X[1])), dmul(F[2], X[2]));
        x1[i] = dadd(dadd(dmul(F[3], X[0]), dmul(F[4], X[1])), dmul(F[5], X[2]));
        x2[i] = dadd(dadd(dmul(F[6], X[0]), dmul(F[7], X[1])), dmul(F[8], X[2]));
    }
    __syncthreads();
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double g0, g1, g2;
        gather_force_fp64(M, rowptr, R.csr0, i, x0, x1, x2, g0, g1, g2);
        acc += dadd(dadd(dmul(g0, g0), dmul(g1, g1)), dmul(g2, g2));
    }
    const double f_aff = dsqrt(block_sum(acc, red));

    // Algorithm 1: displacement BCs on fixed nodes, initial free displacement.
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const bool fixed = i >= nf;
        const double X[3] = {X0[i], X1[i], X2[i]};
        double u[3];
        for (int r = 0; r < 3; ++r) {
            const double xa = r == 0 ? x0[i] : (r == 1 ? x1[i] : x2[i]);
            const double uaff = dsub(xa, X[r]);
            if (fixed || P.init == 1) u[r] = uaff;
            else if (P.init == 2) u[r] = (r == 0 ? u0[i] : (r == 1 ? u1[i] : u2[i]));
            else u[r] = 0.0;
        }
        u0[i] = u[0]; u1[i] = u[1]; u2[i] = u[2];
        if (!fixed) { v0[i] = 0.0; v1[i] = 0.0; v2[i] = 0.0; }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        x0[i] = dadd(X0[i], u0[i]);
        x1[i] = dadd(X1[i], u1[i]);
        x2[i] = dadd(X2[i], u2[i]);
    }
    __syncthreads();
    // getInternalForces(u); update accelerations (free DOFs).
    acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double g0, g1, g2;
        gather_force_fp64(M, rowptr, R.csr0, i, x0, x1, x2, g0, g1, g2);
        acc += dadd(dadd(dmul(g0, g0), dmul(g1, g1)), dmul(g2, g2));
        if (i < nf) {
            const double m = mass[i];
            a0[i] = ddiv(g0, m); a1[i] = ddiv(g1, m); a2[i] = ddiv(g2, m);
        }
    }
    const double f0 = dsqrt(block_sum(acc, red));
    const double f_ref = f_aff > f0 ? f_aff : f0;
    const double thresh = P.tol * f_ref;

    const double dt = dmul(P.alpha, R.dtc);  // compute next time step (constant)
    const double hdt = dmul(0.5, dt);
    const double mc = -R.c;
    int64_t it = 0;
    int status = RVE_MAXITER;
    double r = 0.0, ke = 0.0;
    for (;;) {
        // partial velocity update; update displacements (free DOFs)
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            double vv0 = dadd(v0[i], dmul(hdt, a0[i]));
            double vv1 = dadd(v1[i], dmul(hdt, a1[i]));
            double vv2 = dadd(v2[i], dmul(hdt, a2[i]));
            double uu0 = dadd(u0[i], dmul(dt, vv0));
            double uu1 = dadd(u1[i], dmul(dt, vv1));
            double uu2 = dadd(u2[i], dmul(dt, vv2));
            v0[i] = vv0; v1[i] = vv1; v2[i] = vv2;
            u0[i] = uu0; u1[i] = uu1; u2[i] = uu2;
            x0[i] = dadd(X0[i], uu0);
            x1[i] = dadd(X1[i], uu1);
            x2[i] = dadd(X2[i], uu2);
        }
        __syncthreads();
        // getInternalForces; damping force; residual; accelerations; velocity
        double rs = 0.0, kes = 0.0;
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            double g0, g1, g2;
            gather_force_fp64(M, rowptr, R.csr0, i, x0, x1, x2, g0, g1, g2);
            const double m = mass[i];
            const double cm = dmul(mc, m);
            double vv0 = v0[i], vv1 = v1[i], vv2 = v2[i];
            rs = dadd(rs, dmul(g0, g0));
            rs = dadd(rs, dmul(g1, g1));
            rs = dadd(rs, dmul(g2, g2));
            const double aa0 = ddiv(dadd(g0, dmul(cm, vv0)), m);
            const double aa1 = ddiv(dadd(g1, dmul(cm, vv1)), m);
            const double aa2 = ddiv(dadd(g2, dmul(cm, vv2)), m);
            vv0 = dadd(vv0, dmul(hdt, aa0));
            vv1 = dadd(vv1, dmul(hdt, aa1));
            vv2 = dadd(vv2, dmul(hdt, aa2));
            a0[i] = aa0; a1[i] = aa1; a2[i] = aa2;
            v0[i] = vv0; v1[i] = vv1; v2[i] = vv2;
            if (P.want_ke) kes += 0.5 * m * (vv0 * vv0 + vv1 * vv1 + vv2 * vv2);
        }
        const double rs_tot = block_sum(rs, red);
        if (P.want_ke) ke = block_sum(kes, red);
        r = dsqrt(rs_tot);
        ++it;
        if (!isfinite(r)) { status = RVE_NAN; break; }
        if (r <= thresh) { status = RVE_OK; break; }
        if (it >= P.max_iter) { status = RVE_MAXITER; break; }
    }
    __syncthreads();
    rve_stress(M, R, F, x0, x1, x2, O.sigma + 9 * (int64_t)p, red);
    if (threadIdx.x == 0) {
        O.iters[p] = it;
        O.rel_res[p] = f_ref > 0.0 ? r / f_ref : (r > 0.0 ? INFINITY : 0.0);
        O.status[p] = status;
        O.f_ref[p] = f_ref;
        O.ke[p] = ke;
    }
    __syncthreads();
}

}  // namespace fe2
