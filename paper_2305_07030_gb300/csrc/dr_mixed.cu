// Mixed-precision dynamic relaxation (Algorithm 1) for a batch of RVEs: one CTA
// per RVE, whole loop in one persistent launch.
//
// Phase 1 (lead): the first lead_iters iterations run in FP64 exactly like the
// FP64 kernel. Random fiber networks are not isostatic and can pass bifurcation
// points (Section II); which equilibrium the relaxation settles into is decided
// early in the transient and is sensitive to force errors far below FP32
// rounding, so the lead keeps that choice the reference one.
//
// Phase 2 (FP32 increments): every element force is written as an exact
// increment about a reference state x_ref,
//     t(d_ref + dd) = t(d_ref) + q_ref dd + dq (d_ref + dd),
//     q = N/l = EA (1/L - 1/l),  dq = EA h / (l l_ref (l + l_ref)),
//     h = l^2 - l_ref^2 = 2 d_ref.dd + dd.dd,
// in which every FP32 operation acts on small quantities. The nodal sum of
// t(d_ref) (g_ref) is evaluated in FP64 and refreshed every rebase_every
// iterations, when the FP32 displacement increment du is folded into the FP64
// displacement. Updates (velocity, displacement increment, damping,
// acceleration) are FP32; the residual norm is accumulated per warp in FP32
// (a sum of squares, no cancellation) and across warps in FP64; the
// convergence test and the stress sum are FP64.
#include "dr_device.cuh"

namespace fe2 {

__device__ __forceinline__ double block_sum_f(float v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = (blockDim.x + 31) >> 5;
    if (lane == 0) red[warp] = (double)v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];
    __syncthreads();
    return t;
}

__device__ __forceinline__ int64_t default_lead(int n) {
    return (int64_t)(1000.0 * cbrt((double)n / 512.0));
}

template <bool SM>
__device__ void solve_rve_mixed(const DevMesh &M, const DevState &S, const DevResults &O,
                                const SolveParams &P, int p, unsigned char *smem, double *red) {
    const RveDesc R = M.rve[p];
    const int n = R.n_nodes, nf = R.n_free;
    const int64_t n0 = R.node0;
    const int32_t *rowptr = M.rowptr + R.rp0;
    unsigned char *base = SM ? smem : reinterpret_cast<unsigned char *>(S.pg + 2 * n0);
    // FP64 view (24 B/node) and FP32 view (2 float4 = 32 B/node) of one buffer.
    double *x0 = reinterpret_cast<double *>(base), *x1 = x0 + n, *x2 = x1 + n;
    float4 *Pq = reinterpret_cast<float4 *>(base);  // x_ref (FP32)
    float4 *Qq = Pq + n;                            // du (FP32)
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = P.F[9 * (int64_t)p + k];
    const double *X0 = M.X0 + n0, *X1 = M.X1 + n0, *X2 = M.X2 + n0;
    double *u0 = S.u0 + n0, *u1 = S.u1 + n0, *u2 = S.u2 + n0;
    double *v0 = S.v0 + n0, *v1 = S.v1 + n0, *v2 = S.v2 + n0;
    double *a0 = S.a0 + n0, *a1 = S.a1 + n0, *a2 = S.a2 + n0;
    const double *mass = M.mass + n0;
    const float *inv_m = M.inv_mass_f + n0;
    float *fv = S.fv + 3 * n0, *fa = S.fa + 3 * n0, *fg = S.fg + 3 * n0;  // [3][n] per RVE

    // ---- setup, identical to the FP64 kernel ----
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
    const double dt = dmul(P.alpha, R.dtc);
    const double hdt = dmul(0.5, dt);
    const double mc = -R.c;
    const int64_t lead = P.lead_iters >= 0 ? P.lead_iters : default_lead(n);
    const int K = P.rebase_every > 0 ? P.rebase_every : 512;

    int64_t it = 0;
    int status = RVE_MAXITER;
    double r = 0.0, ke = 0.0;
    bool done = false;

    // ---- phase 1: FP64 lead ----
    while (it < lead) {
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
        if (!isfinite(r)) { status = RVE_NAN; done = true; break; }
        if (r <= thresh) { status = RVE_OK; done = true; break; }
        if (it >= P.max_iter) { status = RVE_MAXITER; done = true; break; }
    }

    // ---- phase 2: FP32 increments about an FP64 reference ----
    if (!done) {
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            fv[i] = (float)v0[i]; fv[n + i] = (float)v1[i]; fv[2 * n + i] = (float)v2[i];
            fa[i] = (float)a0[i]; fa[n + i] = (float)a1[i]; fa[2 * n + i] = (float)a2[i];
        }
        const float hdtf = (float)hdt, dtf = (float)dt, cf = (float)R.c;
        bool rebase = true;
        int since = 0;
        for (;;) {
            if (rebase) {
                // Fold du into u (FP64), stage x = X + u in FP64, g_ref = g(x) in FP64.
                __syncthreads();
                if (it > lead) {
                    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
                        const float4 du = Qq[i];
                        u0[i] = dadd(u0[i], (double)du.x);
                        u1[i] = dadd(u1[i], (double)du.y);
                        u2[i] = dadd(u2[i], (double)du.z);
                    }
                    __syncthreads();
                }
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    x0[i] = dadd(X0[i], u0[i]);
                    x1[i] = dadd(X1[i], u1[i]);
                    x2[i] = dadd(X2[i], u2[i]);
                }
                __syncthreads();
                for (int i = threadIdx.x; i < nf; i += blockDim.x) {
                    double g0, g1, g2;
                    gather_force_fp64(M, rowptr, R.csr0, i, x0, x1, x2, g0, g1, g2);
                    fg[i] = (float)g0; fg[n + i] = (float)g1; fg[2 * n + i] = (float)g2;
                }
                __syncthreads();
                // Re-stage as FP32 reference positions and zero increments.
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const float4 xr = make_float4((float)dadd(X0[i], u0[i]), (float)dadd(X1[i], u1[i]),
                                                  (float)dadd(X2[i], u2[i]), 0.f);
                    // x0..x2 alias Pq/Qq: read everything of node i above first.
                    Pq[i] = xr;
                    Qq[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                __syncthreads();
                rebase = false;
                since = 0;
            }
            // partial velocity update; update displacement increments
            for (int i = threadIdx.x; i < nf; i += blockDim.x) {
                float w0 = fv[i] + hdtf * fa[i];
                float w1 = fv[n + i] + hdtf * fa[n + i];
                float w2 = fv[2 * n + i] + hdtf * fa[2 * n + i];
                fv[i] = w0; fv[n + i] = w1; fv[2 * n + i] = w2;
                float4 du = Qq[i];
                du.x += dtf * w0; du.y += dtf * w1; du.z += dtf * w2;
                Qq[i] = du;
            }
            __syncthreads();
            // forces as FP32 increments; damping; residual; accelerations; velocity
            float rs = 0.f, kes = 0.f;
            for (int i = threadIdx.x; i < nf; i += blockDim.x) {
                const float4 pi = Pq[i], qi = Qq[i];
                float g0 = fg[i], g1 = fg[n + i], g2 = fg[2 * n + i];
                const int beg = rowptr[i], end = rowptr[i + 1];
                for (int k = beg; k < end; ++k) {
                    const int64_t kk = R.csr0 + k;
                    const int j = M.col[kk];
                    const float2 ei = M.EAf_invLf[kk];
                    const float4 pj = Pq[j], qj = Qq[j];
                    const float r0 = pj.x - pi.x, r1 = pj.y - pi.y, r2 = pj.z - pi.z;
                    const float e0 = qj.x - qi.x, e1 = qj.y - qi.y, e2 = qj.z - qi.z;
                    const float lr2 = r0 * r0 + r1 * r1 + r2 * r2;
                    const float ril = rsqrtf(lr2);
                    const float lr = lr2 * ril;
                    const float qref = ei.x * (ei.y - ril);
                    const float h = 2.f * (r0 * e0 + r1 * e1 + r2 * e2) + (e0 * e0 + e1 * e1 + e2 * e2);
                    const float rl = rsqrtf(lr2 + h);
                    const float l = (lr2 + h) * rl;
                    const float dq = __fdividef(ei.x * h * rl * ril, l + lr);
                    g0 += qref * e0 + dq * (r0 + e0);
                    g1 += qref * e1 + dq * (r1 + e1);
                    g2 += qref * e2 + dq * (r2 + e2);
                }
                const float im = inv_m[i];
                float w0 = fv[i], w1 = fv[n + i], w2 = fv[2 * n + i];
                const float aa0 = g0 * im - cf * w0;
                const float aa1 = g1 * im - cf * w1;
                const float aa2 = g2 * im - cf * w2;
                w0 += hdtf * aa0; w1 += hdtf * aa1; w2 += hdtf * aa2;
                fa[i] = aa0; fa[n + i] = aa1; fa[2 * n + i] = aa2;
                fv[i] = w0; fv[n + i] = w1; fv[2 * n + i] = w2;
                rs += g0 * g0 + g1 * g1 + g2 * g2;
                if (P.want_ke) kes += (w0 * w0 + w1 * w1 + w2 * w2) * (0.5f / im);
            }
            const double rs_tot = block_sum_f(rs, red);
            if (P.want_ke) ke = block_sum_f(kes, red);
            r = sqrt(rs_tot);
            ++it;
            ++since;
            if (!isfinite(r)) { status = RVE_NAN; break; }
            if (r <= thresh) { status = RVE_OK; break; }
            if (it >= P.max_iter) { status = RVE_MAXITER; break; }
            if (since >= K) rebase = true;
        }
        // Final displacement u = u_ref + du (FP64) and FP64 positions for the stress.
        for (int i = threadIdx.x; i < nf; i += blockDim.x) {
            const float4 du = Qq[i];
            u0[i] = dadd(u0[i], (double)du.x);
            u1[i] = dadd(u1[i], (double)du.y);
            u2[i] = dadd(u2[i], (double)du.z);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            x0[i] = dadd(X0[i], u0[i]);
            x1[i] = dadd(X1[i], u1[i]);
            x2[i] = dadd(X2[i], u2[i]);
        }
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

template <bool SM>
__global__ void __launch_bounds__(512) dr_mixed_kernel(DevMesh M, DevState S, DevResults O,
                                                        SolveParams P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= P.queue_len) return;
        solve_rve_mixed<SM>(M, S, O, P, P.queue[item], smem_raw, red);
    }
}

int launch_dr_mixed(const DevMesh &m, const DevState &s, const DevResults &r, const SolveParams &p,
                    int grid, int block, size_t smem, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p.smem_positions) {
        cudaFuncSetAttribute(dr_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        dr_mixed_kernel<true><<<grid, block, smem, st>>>(m, s, r, p);
    } else {
        dr_mixed_kernel<false><<<grid, block, 0, st>>>(m, s, r, p);
    }
    return (int)cudaGetLastError();
}

int occupancy_dr_mixed(int smem_positions, int block, size_t smem) {
    int n = 0;
    if (smem_positions) {
        cudaFuncSetAttribute(dr_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dr_mixed_kernel<true>, block, smem);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dr_mixed_kernel<false>, block, 0);
    }
    return n;
}

}  // namespace fe2
