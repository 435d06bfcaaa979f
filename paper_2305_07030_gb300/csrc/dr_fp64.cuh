// FP64 oracle-order solve of one RVE by one CTA (Algorithm 1), shared by the
// persistent batch kernel and the allocation-free single-RVE entry point.
#pragma once
#include "dr_device.cuh"

namespace fe2 {

// Force of every element with a free end on its first node (caller
// orientation a -> b): t_e = (N/l) d, d = x_b - x_a, in the operations of
// gather_force_fp64. Node b's gather would compute d' = -d exactly, the same
// l, N and q, and q d' = -t_e exactly, so summing +-t_e in a node's row order
// reproduces its gather bit for bit with half the square roots and divisions.
__device__ __forceinline__ void element_forces_fp64(const DevMesh &M, const RveDesc &R, int nf,
                                                    const double *x0, const double *x1,
                                                    const double *x2, double *tf) {
    for (int e = threadIdx.x; e < R.n_elems; e += blockDim.x) {
        const int64_t ee = R.elem0 + e;
        const int a = M.el_a[ee], b = M.el_b[ee];
        if (a >= nf && b >= nf) continue;  // both ends fixed: no free node needs it
        const double d0 = dsub(x0[b], x0[a]), d1 = dsub(x1[b], x1[a]), d2 = dsub(x2[b], x2[a]);
        const double l = dsqrt(dadd(dadd(dmul(d0, d0), dmul(d1, d1)), dmul(d2, d2)));
        const double N = dmul(M.el_EA[ee], dsub(ddiv(l, M.el_L[ee]), 1.0));
        const double q = ddiv(N, l);
        double *t = tf + 3 * ee;
        t[0] = dmul(q, d0);
        t[1] = dmul(q, d1);
        t[2] = dmul(q, d2);
    }
}

// Node i's internal force from the element forces, in its CSR row order.
__device__ __forceinline__ void gather_table_fp64(const DevMesh &M, const RveDesc &R,
                                                  const int32_t *rowptr, int i, const double *tf,
                                                  double &g0, double &g1, double &g2) {
    const int beg = rowptr[i], end = rowptr[i + 1];
    const double *tr = tf + 3 * R.elem0;
    g0 = 0.0; g1 = 0.0; g2 = 0.0;
    for (int k = beg; k < end; ++k) {
        const int w = M.csr_el[R.csr0 + k];
        const double *t = tr + 3 * (w >> 1);
        if (w & 1) {
            g0 = dsub(g0, t[0]); g1 = dsub(g1, t[1]); g2 = dsub(g2, t[2]);
        } else {
            g0 = dadd(g0, t[0]); g1 = dadd(g1, t[1]); g2 = dadd(g2, t[2]);
        }
    }
}

// ET: element forces through the per-element table S.tf (batched path);
// otherwise every directed edge is evaluated by gather_force_fp64.
template <bool SM, bool ET>
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
    // Energy check (want_ke == 2, Algorithm 1's optional energy balance): per
    // free DOF the previous internal force gp and damping force fp, and the
    // trapezoid sums of this step's increment du = dt v^(n-1/2) against them.
    const bool energy = P.want_ke == 2;
    double *gp0 = nullptr, *gp1 = nullptr, *gp2 = nullptr, *fp0 = nullptr, *fp1 = nullptr, *fp2 = nullptr;
    if (energy) {
        gp0 = S.gp + 3 * n0; gp1 = gp0 + n; gp2 = gp1 + n;
        fp0 = S.fdp + 3 * n0; fp1 = fp0 + n; fp2 = fp1 + n;
    }
    acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double g0, g1, g2;
        gather_force_fp64(M, rowptr, R.csr0, i, x0, x1, x2, g0, g1, g2);
        acc += dadd(dadd(dmul(g0, g0), dmul(g1, g1)), dmul(g2, g2));
        if (i < nf) {
            const double m = mass[i];
            a0[i] = ddiv(g0, m); a1[i] = ddiv(g1, m); a2[i] = ddiv(g2, m);
            if (energy) {
                // the work sums start from the initial force and no damping force
                gp0[i] = g0; gp1[i] = g1; gp2[i] = g2;
                fp0[i] = 0.0; fp1[i] = 0.0; fp2[i] = 0.0;
            }
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
    double r = 0.0, ke = 0.0, wint = 0.0, wext = 0.0;
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
        if (ET) {
            element_forces_fp64(M, R, nf, x0, x1, x2, S.tf);
            __syncthreads();
        }
        // getInternalForces; damping force; residual; accelerations; velocity
        double rs = 0.0, kes = 0.0, wis = 0.0, wes = 0.0;
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            double g0, g1, g2;
            if (ET) gather_table_fp64(M, R, rowptr, i, S.tf, g0, g1, g2);
            else gather_force_fp64(M, rowptr, R.csr0, i, x0, x1, x2, g0, g1, g2);
            const double m = mass[i];
            const double cm = dmul(mc, m);
            double vv0 = v0[i], vv1 = v1[i], vv2 = v2[i];
            rs = dadd(rs, dmul(g0, g0));
            rs = dadd(rs, dmul(g1, g1));
            rs = dadd(rs, dmul(g2, g2));
            if (energy) {
                const double f0 = dmul(cm, vv0), f1 = dmul(cm, vv1), f2 = dmul(cm, vv2);
                const double du0 = dmul(dt, vv0), du1 = dmul(dt, vv1), du2 = dmul(dt, vv2);
                wis = dadd(wis, dmul(du0, dadd(gp0[i], g0)));
                wis = dadd(wis, dmul(du1, dadd(gp1[i], g1)));
                wis = dadd(wis, dmul(du2, dadd(gp2[i], g2)));
                wes = dadd(wes, dmul(du0, dadd(fp0[i], f0)));
                wes = dadd(wes, dmul(du1, dadd(fp1[i], f1)));
                wes = dadd(wes, dmul(du2, dadd(fp2[i], f2)));
                gp0[i] = g0; gp1[i] = g1; gp2[i] = g2;
                fp0[i] = f0; fp1[i] = f1; fp2[i] = f2;
            }
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
        if (energy) {
            wint = dsub(wint, dmul(0.5, block_sum(wis, red)));
            wext = dadd(wext, dmul(0.5, block_sum(wes, red)));
        }
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
        if (O.wint) O.wint[p] = wint;
        if (O.wext) O.wext[p] = wext;
    }
    __syncthreads();
}

}  // namespace fe2
