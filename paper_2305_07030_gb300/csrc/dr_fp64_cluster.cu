// FP64 dynamic relaxation (Algorithm 1) of one RVE on a thread-block cluster.
//
// The single-CTA FP64 kernel (dr_fp64.cu) is bound by one SM's FP64 pipe:
// an RVE of a few thousand nodes needs hundreds of microseconds per
// iteration there. This kernel spreads an RVE over the CTAs of a cluster, one
// spatial part each (the parts of the batch layout), so the RVE's arithmetic
// runs on as many SMs. The paper used one team per sub-problem (Section III);
// a cluster is a team that spans SMs.
//
// Arithmetic is the single-CTA kernel's, operation for operation, so the
// trajectory is the oracle's bit for bit:
//  * each CTA keeps its own nodes' positions in shared memory (two buffers,
//    one per evaluation parity) and reads neighbours of other parts through
//    distributed shared memory;
//  * each element with an end among the CTA's free nodes has a slot in the
//    CTA's element table; its force on the first end is evaluated once per
//    iteration with the operations of element_forces_fp64;
//  * each free node sums the +- slot forces of its CSR row in row order, then
//    the damping, acceleration and velocity updates follow as in the
//    single-CTA kernel;
//  * one cluster barrier per iteration. The partial sums of the residual
//    (and the energy terms) of evaluation n are published before the barrier
//    that makes evaluation n+1's positions visible, and every CTA totals them
//    in rank order after it, so the test of evaluation n runs one update
//    later; the displacement alternates between two buffers so that the
//    stopping evaluation's state is still intact.
// The residual and energy sums are associated differently from the oracle's
// serial sums (per CTA, then across the cluster), as in the single-CTA
// kernel's block sums.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "dr_device.cuh"

namespace cg = cooperative_groups;

namespace fe2 {

namespace {

struct Fp64ClusterShared {
    double part[2][4];               // this CTA's sums of evaluation n (parity n & 1):
                                     // squared residual, kinetic energy, work terms
    const double *partp[kMaxParts];  // every CTA's `part`
    const double *xp[2][kMaxParts];  // every CTA's position buffers
    double red[32];                  // block reductions
    int item;
};

// A neighbour's position component: (part << 16 | index) into the cluster's
// shared-memory buffer `buf` ([3][part_cap] doubles per CTA).
__device__ __forceinline__ const double *pos_of(const Fp64ClusterShared &sh, int buf, int ref, int part_cap) {
    return sh.xp[buf][ref >> 16] + (ref & 0xffff);
}

// Net internal force on own node gi (RVE-local id) by the per-edge gather of
// gather_force_fp64, neighbours read through the cluster (set-up only).
__device__ __forceinline__ void gather_force_cluster(const DevMesh &M, const RveDesc &R,
                                                     const Fp64ClusterShared &sh, int buf, int part_cap,
                                                     const int32_t *rowptr, int gi, int me, int k,
                                                     double &g0, double &g1, double &g2) {
    const int beg = rowptr[gi], end = rowptr[gi + 1];
    const double *xi = sh.xp[buf][me] + k;
    const double xi0 = xi[0], xi1 = xi[part_cap], xi2 = xi[2 * part_cap];
    g0 = 0.0; g1 = 0.0; g2 = 0.0;
    for (int q = beg; q < end; ++q) {
        const int64_t kk = R.csr0 + q;
        const double *xj = pos_of(sh, buf, M.col_part[kk], part_cap);
        const double d0 = dsub(xj[0], xi0), d1 = dsub(xj[part_cap], xi1), d2 = dsub(xj[2 * part_cap], xi2);
        const double l = dsqrt(dadd(dadd(dmul(d0, d0), dmul(d1, d1)), dmul(d2, d2)));
        const double N = dmul(M.EA[kk], dsub(ddiv(l, M.L[kk]), 1.0));
        const double q2 = ddiv(N, l);
        g0 = dadd(g0, dmul(q2, d0));
        g1 = dadd(g1, dmul(q2, d1));
        g2 = dadd(g2, dmul(q2, d2));
    }
}

// Sum over the cluster of one published value (rank order, same bits in
// every CTA). Call after a cluster barrier that follows the publication.
__device__ __forceinline__ double cluster_value(const Fp64ClusterShared &sh, int C, int parity, int field) {
    double t = 0.0;
    for (int r = 0; r < C; ++r) t = dadd(t, sh.partp[r][parity * 4 + field]);
    return t;
}

__device__ __forceinline__ void cl_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cl_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

}  // namespace

// One RVE on the cluster. XB (smem) is this CTA's [2][3][part_cap] position
// buffers; T the element table, [3][slot_cap] in shared memory (TSM) or this
// part's region of the global table. With SSM the own free nodes' state lives
// in shared memory too (ST: displacement [2][3][free_cap], velocity and
// acceleration [3][free_cap] each, mass [free_cap]); otherwise in global
// memory (L2).
template <bool TSM, bool SSM>
__device__ void solve_rve_fp64_cluster(cg::cluster_group &cl, Fp64ClusterShared &sh, const DevMesh &M,
                                       const DevState &S, const DevResults &O, const SolveParams &P, int p,
                                       double *XB, double *ST, double *Tsm, int part_cap, int free_cap,
                                       int slot_cap) {
    const RveDesc R = M.rve[p];
    const int me = (int)cl.block_rank(), C = (int)cl.num_blocks();
    const int32_t *po = M.part_off + (int64_t)p * 2 * (kMaxParts + 1);
    const int n = R.n_nodes, nf = R.n_free;
    const int f0 = po[me], nfr = po[me + 1] - f0;
    const int g0 = po[kMaxParts + 1 + me], nfx = po[kMaxParts + 1 + me + 1] - g0;
    const int m = nfr + nfx;
    auto gidx = [&](int k) { return k < nfr ? f0 + k : nf + g0 + (k - nfr); };
    const int64_t n0 = R.node0;
    const int32_t *rowptr = M.rowptr + R.rp0;
    const int32_t *ps = M.fp_part_slot + (int64_t)p * (kMaxParts + 1);
    const int s0 = ps[me], ns = ps[me + 1] - s0;
    const int4 *slots = M.fp_slot + R.slot0 + s0;
    const int tstride = TSM ? slot_cap : ns;
    double *T = TSM ? Tsm : S.fpt + 3 * (R.slot0 + s0);
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = P.F[9 * (int64_t)p + k];
    const double *X0 = M.X0 + n0, *X1 = M.X1 + n0, *X2 = M.X2 + n0;
    // displacement buffers: even evaluations in the output arrays, odd ones
    // in the alternate [3][n] block (selected per iteration, no indexed arrays)
    double *const ue0 = S.u0 + n0, *const ue1 = S.u1 + n0, *const ue2 = S.u2 + n0;
    double *const uo0 = S.ualt + 3 * n0, *const uo1 = uo0 + n, *const uo2 = uo1 + n;
    // free-node state, addressed by the RVE-local node id i = f0 + k: shared
    // arrays are offset by -f0 so that the same index serves both places
    double *v0 = S.v0 + n0, *v1 = S.v1 + n0, *v2 = S.v2 + n0;
    double *a0 = S.a0 + n0, *a1 = S.a1 + n0, *a2 = S.a2 + n0;
    const double *mass = M.mass + n0;
    double *su[2][3] = {};
    if (SSM) {
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 3; ++c) su[b][c] = ST + (3 * b + c) * free_cap - f0;
        double *sv = ST + 6 * free_cap - f0;
        v0 = sv; v1 = sv + free_cap; v2 = sv + 2 * free_cap;
        double *sa = ST + 9 * free_cap - f0;
        a0 = sa; a1 = sa + free_cap; a2 = sa + 2 * free_cap;
        double *sm = ST + 12 * free_cap - f0;
        for (int k = threadIdx.x; k < nfr; k += blockDim.x) sm[f0 + k] = M.mass[n0 + f0 + k];
        mass = sm;
    }
    double *const x0b = XB, *const x1b = XB + 3 * part_cap;
    const bool energy = P.want_ke == 2;
    double *gp0 = nullptr, *gp1 = nullptr, *gp2 = nullptr, *fp0 = nullptr, *fp1 = nullptr, *fp2 = nullptr;
    if (energy) {
        gp0 = S.gp + 3 * n0; gp1 = gp0 + n; gp2 = gp1 + n;
        fp0 = S.fdp + 3 * n0; fp1 = fp0 + n; fp2 = fp1 + n;
    }

    // f_ref, part 1: forces in the affine configuration x = F X (all DOFs)
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int i = gidx(k);
        const double Xv[3] = {X0[i], X1[i], X2[i]};
        x0b[k] = dadd(dadd(dmul(F[0], Xv[0]), dmul(F[1], Xv[1])), dmul(F[2], Xv[2]));
        x0b[part_cap + k] = dadd(dadd(dmul(F[3], Xv[0]), dmul(F[4], Xv[1])), dmul(F[5], Xv[2]));
        x0b[2 * part_cap + k] = dadd(dadd(dmul(F[6], Xv[0]), dmul(F[7], Xv[1])), dmul(F[8], Xv[2]));
    }
    cl.sync();
    double acc = 0.0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        double g0v, g1v, g2v;
        gather_force_cluster(M, R, sh, 0, part_cap, rowptr, gidx(k), me, k, g0v, g1v, g2v);
        acc += dadd(dadd(dmul(g0v, g0v), dmul(g1v, g1v)), dmul(g2v, g2v));
    }
    {
        const double t = block_sum(acc, sh.red);
        if (threadIdx.x == 0) sh.part[0][0] = t;
    }
    cl.sync();  // every CTA's sum published; every gather of x_aff done
    const double f_aff = dsqrt(cluster_value(sh, C, 0, 0));

    // Algorithm 1: displacement BCs on fixed nodes, initial free displacement
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int i = gidx(k);
        const bool fixed = k >= nfr;
        const double Xv[3] = {X0[i], X1[i], X2[i]};
        double u[3];
        for (int r = 0; r < 3; ++r) {
            const double uaff = dsub(x0b[r * part_cap + k], Xv[r]);
            if (fixed || P.init == 1) u[r] = uaff;
            else if (P.init == 2) u[r] = r == 0 ? ue0[i] : (r == 1 ? ue1[i] : ue2[i]);
            else u[r] = 0.0;
        }
        ue0[i] = u[0]; ue1[i] = u[1]; ue2[i] = u[2];
        if (SSM) {
            if (!fixed)
                for (int c = 0; c < 3; ++c) { su[0][c][i] = u[c]; su[1][c][i] = u[c]; }
        } else {
            uo0[i] = u[0]; uo1[i] = u[1]; uo2[i] = u[2];
        }
        for (int r = 0; r < 3; ++r) {
            const double xv = dadd(Xv[r], u[r]);
            x0b[r * part_cap + k] = xv;
            x1b[r * part_cap + k] = xv;  // fixed positions live in both buffers
        }
        if (!fixed) { v0[i] = 0.0; v1[i] = 0.0; v2[i] = 0.0; }
    }
    cl.sync();
    // getInternalForces(u); update accelerations (free DOFs)
    acc = 0.0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int i = gidx(k);
        double g0v, g1v, g2v;
        gather_force_cluster(M, R, sh, 0, part_cap, rowptr, i, me, k, g0v, g1v, g2v);
        acc += dadd(dadd(dmul(g0v, g0v), dmul(g1v, g1v)), dmul(g2v, g2v));
        if (k < nfr) {
            const double mm = mass[i];
            a0[i] = ddiv(g0v, mm); a1[i] = ddiv(g1v, mm); a2[i] = ddiv(g2v, mm);
            if (energy) {
                gp0[i] = g0v; gp1[i] = g1v; gp2[i] = g2v;
                fp0[i] = 0.0; fp1[i] = 0.0; fp2[i] = 0.0;
            }
        }
    }
    {
        const double t = block_sum(acc, sh.red);
        if (threadIdx.x == 0) sh.part[1][0] = t;
    }
    cl.sync();
    const double f0v = dsqrt(cluster_value(sh, C, 1, 0));
    const double f_ref = f_aff > f0v ? f_aff : f0v;
    const double thresh = P.tol * f_ref;
    const double dt = dmul(P.alpha, R.dtc);  // compute next time step (constant)
    const double hdt = dmul(0.5, dt);
    const double mc = -R.c;
    int64_t it = 0;
    int status = RVE_MAXITER;
    double r = 0.0, ke = 0.0, wint = 0.0, wext = 0.0;
    for (;;) {
        const int cb = (int)((it + 1) & 1);  // buffers of evaluation it + 1
        const int pb = cb ^ 1;               // ... and of evaluation it
        double *un0, *un1, *un2;
        const double *up0, *up1, *up2;
        if (SSM) {
            un0 = cb ? su[1][0] : su[0][0]; un1 = cb ? su[1][1] : su[0][1]; un2 = cb ? su[1][2] : su[0][2];
            up0 = cb ? su[0][0] : su[1][0]; up1 = cb ? su[0][1] : su[1][1]; up2 = cb ? su[0][2] : su[1][2];
        } else {
            un0 = cb ? uo0 : ue0; un1 = cb ? uo1 : ue1; un2 = cb ? uo2 : ue2;
            up0 = cb ? ue0 : uo0; up1 = cb ? ue1 : uo1; up2 = cb ? ue2 : uo2;
        }
        double *const xc = cb ? XB + 3 * part_cap : XB;
        // partial velocity update; update displacements (own free DOFs)
        for (int k = threadIdx.x; k < nfr; k += blockDim.x) {
            const int i = f0 + k;
            const double vv0 = dadd(v0[i], dmul(hdt, a0[i]));
            const double vv1 = dadd(v1[i], dmul(hdt, a1[i]));
            const double vv2 = dadd(v2[i], dmul(hdt, a2[i]));
            const double uu0 = dadd(up0[i], dmul(dt, vv0));
            const double uu1 = dadd(up1[i], dmul(dt, vv1));
            const double uu2 = dadd(up2[i], dmul(dt, vv2));
            v0[i] = vv0; v1[i] = vv1; v2[i] = vv2;
            un0[i] = uu0; un1[i] = uu1; un2[i] = uu2;
            xc[k] = dadd(X0[i], uu0);
            xc[part_cap + k] = dadd(X1[i], uu1);
            xc[2 * part_cap + k] = dadd(X2[i], uu2);
        }
        // one barrier: positions of evaluation it + 1 and the sums of
        // evaluation it become visible to the whole cluster
        cl_arrive();
        cl_wait();
        if (it > 0) {
            const double rs = cluster_value(sh, C, pb, 0);
            if (P.want_ke) ke = cluster_value(sh, C, pb, 1);
            if (energy) {
                wint = dsub(wint, dmul(0.5, cluster_value(sh, C, pb, 2)));
                wext = dadd(wext, dmul(0.5, cluster_value(sh, C, pb, 3)));
            }
            r = dsqrt(rs);
            if (!isfinite(r)) { status = RVE_NAN; break; }
            if (r <= thresh) { status = RVE_OK; break; }
            if (it >= P.max_iter) { status = RVE_MAXITER; break; }
        }
        // element forces of the CTA's slots at evaluation it + 1
        for (int s = threadIdx.x; s < ns; s += blockDim.x) {
            const int4 sl = slots[s];
            const int64_t ee = R.elem0 + sl.x;
            const double *xa = pos_of(sh, cb, sl.y, part_cap), *xb = pos_of(sh, cb, sl.z, part_cap);
            const double d0 = dsub(xb[0], xa[0]);
            const double d1 = dsub(xb[part_cap], xa[part_cap]);
            const double d2 = dsub(xb[2 * part_cap], xa[2 * part_cap]);
            const double l = dsqrt(dadd(dadd(dmul(d0, d0), dmul(d1, d1)), dmul(d2, d2)));
            const double N = dmul(M.el_EA[ee], dsub(ddiv(l, M.el_L[ee]), 1.0));
            const double q = ddiv(N, l);
            T[s] = dmul(q, d0);
            T[tstride + s] = dmul(q, d1);
            T[2 * tstride + s] = dmul(q, d2);
        }
        __syncthreads();
        // getInternalForces (slot sums in row order); damping force; residual;
        // accelerations; velocity (own free DOFs)
        double rs = 0.0, kes = 0.0, wis = 0.0, wes = 0.0;
        for (int k = threadIdx.x; k < nfr; k += blockDim.x) {
            const int i = f0 + k;
            const int beg = rowptr[i], end = rowptr[i + 1];
            double g0v = 0.0, g1v = 0.0, g2v = 0.0;
            for (int q = beg; q < end; ++q) {
                const int w = M.fp_csr_slot[R.csr0 + q];
                const int sl = w >> 1;
                if (w & 1) {
                    g0v = dsub(g0v, T[sl]); g1v = dsub(g1v, T[tstride + sl]); g2v = dsub(g2v, T[2 * tstride + sl]);
                } else {
                    g0v = dadd(g0v, T[sl]); g1v = dadd(g1v, T[tstride + sl]); g2v = dadd(g2v, T[2 * tstride + sl]);
                }
            }
            const double mm = mass[i];
            const double cm = dmul(mc, mm);
            double vv0 = v0[i], vv1 = v1[i], vv2 = v2[i];
            rs = dadd(rs, dmul(g0v, g0v));
            rs = dadd(rs, dmul(g1v, g1v));
            rs = dadd(rs, dmul(g2v, g2v));
            if (energy) {
                const double e0 = dmul(cm, vv0), e1 = dmul(cm, vv1), e2 = dmul(cm, vv2);
                const double du0 = dmul(dt, vv0), du1 = dmul(dt, vv1), du2 = dmul(dt, vv2);
                wis = dadd(wis, dmul(du0, dadd(gp0[i], g0v)));
                wis = dadd(wis, dmul(du1, dadd(gp1[i], g1v)));
                wis = dadd(wis, dmul(du2, dadd(gp2[i], g2v)));
                wes = dadd(wes, dmul(du0, dadd(fp0[i], e0)));
                wes = dadd(wes, dmul(du1, dadd(fp1[i], e1)));
                wes = dadd(wes, dmul(du2, dadd(fp2[i], e2)));
                gp0[i] = g0v; gp1[i] = g1v; gp2[i] = g2v;
                fp0[i] = e0; fp1[i] = e1; fp2[i] = e2;
            }
            const double aa0 = ddiv(dadd(g0v, dmul(cm, vv0)), mm);
            const double aa1 = ddiv(dadd(g1v, dmul(cm, vv1)), mm);
            const double aa2 = ddiv(dadd(g2v, dmul(cm, vv2)), mm);
            vv0 = dadd(vv0, dmul(hdt, aa0));
            vv1 = dadd(vv1, dmul(hdt, aa1));
            vv2 = dadd(vv2, dmul(hdt, aa2));
            a0[i] = aa0; a1[i] = aa1; a2[i] = aa2;
            v0[i] = vv0; v1[i] = vv1; v2[i] = vv2;
            if (P.want_ke) kes += 0.5 * mm * (vv0 * vv0 + vv1 * vv1 + vv2 * vv2);
        }
        // this CTA's sums of evaluation it + 1, totalled after the next barrier
        {
            const double t0 = block_sum(rs, sh.red);
            const double t1 = P.want_ke ? block_sum(kes, sh.red) : 0.0;
            const double t2 = energy ? block_sum(wis, sh.red) : 0.0;
            const double t3 = energy ? block_sum(wes, sh.red) : 0.0;
            if (threadIdx.x == 0) {
                sh.part[cb][0] = t0;
                sh.part[cb][1] = t1;
                sh.part[cb][2] = t2;
                sh.part[cb][3] = t3;
            }
        }
        ++it;
    }
    // The stopping evaluation is `it`: its displacement is in ub[it & 1] and
    // its positions in x[it & 1]. Final displacement to the output buffer,
    // positions of every own node to the global scratch for the stress sum.
    const int fb = (int)(it & 1);
    const double *const xf = fb ? XB + 3 * part_cap : XB;
    double *xg = S.xg + 3 * n0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int i = gidx(k);
        if (SSM && k < nfr) {
            ue0[i] = fb ? su[1][0][i] : su[0][0][i];
            ue1[i] = fb ? su[1][1][i] : su[0][1][i];
            ue2[i] = fb ? su[1][2][i] : su[0][2][i];
        } else if (!SSM && fb == 1 && k < nfr) {
            ue0[i] = uo0[i]; ue1[i] = uo1[i]; ue2[i] = uo2[i];
        }
        xg[i] = xf[k];
        xg[n + i] = xf[part_cap + k];
        xg[2 * n + i] = xf[2 * part_cap + k];
    }
    __threadfence();
    cl.sync();
    if (me == 0) rve_stress(M, R, F, xg, xg + n, xg + 2 * n, O.sigma + 9 * (int64_t)p, sh.red);
    if (me == 0 && threadIdx.x == 0) {
        O.iters[p] = it;
        O.rel_res[p] = f_ref > 0.0 ? r / f_ref : (r > 0.0 ? INFINITY : 0.0);
        O.status[p] = status;
        O.f_ref[p] = f_ref;
        O.ke[p] = ke;
        if (O.wint) O.wint[p] = wint;
        if (O.wext) O.wext[p] = wext;
    }
    cl.sync();  // the next RVE may overwrite the buffers
}

template <bool TSM, bool SSM>
__global__ void __launch_bounds__(512, 1) dr_fp64_cluster_kernel(DevMesh M, DevState S, DevResults O,
                                                                 SolveParams P, int part_cap, int free_cap,
                                                                 int slot_cap) {
    extern __shared__ __align__(16) double dsm_fp64[];
    __shared__ Fp64ClusterShared sh;
    cg::cluster_group cl = cg::this_cluster();
    double *XB = dsm_fp64;                               // [2][3][part_cap]
    double *ST = dsm_fp64 + 6 * part_cap;                // free-node state when SSM
    double *T = ST + (SSM ? 13 * (size_t)free_cap : 0);  // [3][slot_cap] when TSM
    const int C = (int)cl.num_blocks();
    if ((int)threadIdx.x < C) {
        const int r = threadIdx.x;
        sh.partp[r] = cl.map_shared_rank(&sh.part[0][0], r);
        sh.xp[0][r] = cl.map_shared_rank(XB, r);
        sh.xp[1][r] = cl.map_shared_rank(XB + 3 * part_cap, r);
    }
    for (;;) {
        if (cl.block_rank() == 0 && threadIdx.x == 0) sh.item = atomicAdd(P.counter, 1);
        cl.sync();
        const int item = *cl.map_shared_rank(&sh.item, 0);
        cl.sync();
        if (item >= P.queue_len) return;
        solve_rve_fp64_cluster<TSM, SSM>(cl, sh, M, S, O, P, P.queue[item], XB, ST, T, part_cap, free_cap,
                                         slot_cap);
    }
}

namespace {
using Fp64ClusterKernel = void (*)(DevMesh, DevState, DevResults, SolveParams, int, int, int);

Fp64ClusterKernel pick_fp64_cluster(bool tsm, bool ssm) {
    if (tsm) return ssm ? dr_fp64_cluster_kernel<true, true> : dr_fp64_cluster_kernel<true, false>;
    return ssm ? dr_fp64_cluster_kernel<false, true> : dr_fp64_cluster_kernel<false, false>;
}

cudaLaunchConfig_t fp64_cluster_config(int clusters, int parts, int block, size_t smem,
                                       cudaLaunchAttribute *attr, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(clusters * parts, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = parts;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// Raise the kernel's dynamic shared-memory limit (and allow 16-CTA
// clusters) once per device and size, so that launches recorded into a CUDA
// graph make no attribute calls of their own.
std::mutex g_fp64c_mutex;
std::map<std::pair<const void *, int>, int> g_fp64c_bytes;

void prepare_fp64_cluster(Fp64ClusterKernel k, size_t smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_fp64c_mutex);
    int &have = g_fp64c_bytes[{reinterpret_cast<const void *>(k), dev}];
    if (have == 0 || have < (int)smem) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        have = std::max(have, (int)smem);
    }
}
}  // namespace

size_t fp64_cluster_smem(int part_cap, int free_cap, int slot_cap, bool tsm, bool ssm) {
    return sizeof(double) * (6 * (size_t)part_cap + (ssm ? 13 * (size_t)free_cap : 0) +
                             (tsm ? 3 * (size_t)slot_cap : 0));
}

int launch_dr_fp64_cluster(const DevMesh &m, const DevState &s, const DevResults &r, const SolveParams &p,
                           int clusters, int parts, int block, int part_cap, int free_cap, int slot_cap,
                           bool tsm, bool ssm, void *stream) {
    cudaLaunchAttribute attr[1];
    const size_t smem = fp64_cluster_smem(part_cap, free_cap, slot_cap, tsm, ssm);
    cudaLaunchConfig_t cfg = fp64_cluster_config(clusters, parts, block, smem, attr,
                                                 static_cast<cudaStream_t>(stream));
    const Fp64ClusterKernel k = pick_fp64_cluster(tsm, ssm);
    prepare_fp64_cluster(k, smem);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, k, m, s, r, p, part_cap, free_cap, slot_cap);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaGetLastError();
}

int occupancy_dr_fp64_cluster(int parts, int block, int part_cap, int free_cap, int slot_cap, bool tsm,
                              bool ssm) {
    cudaLaunchAttribute attr[1];
    const size_t smem = fp64_cluster_smem(part_cap, free_cap, slot_cap, tsm, ssm);
    cudaLaunchConfig_t cfg = fp64_cluster_config(parts * 64, parts, block, smem, attr, nullptr);
    const Fp64ClusterKernel k = pick_fp64_cluster(tsm, ssm);
    prepare_fp64_cluster(k, smem);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace fe2
