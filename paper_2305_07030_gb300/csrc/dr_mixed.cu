// Mixed-precision dynamic relaxation (Algorithm 1) for a batch of RVEs: one
// thread-block cluster per RVE, whole loop inside one persistent launch.
//
// Layout. The RVE is split spatially into `parts` pieces, one per CTA of the
// cluster; a CTA stages the current positions of its own nodes in its shared
// memory and reads neighbours owned by other CTAs through distributed shared
// memory. The paper used one thread team per sub-problem (Section III); a
// cluster lets one sub-problem span several SMs when one team is not enough.
//
// Precision. All arithmetic runs on the FP32 pipes (GB300's FP64 rate is a
// small fraction of FP32):
//  * lead phase: double-float (hi + lo FP32 pairs, ~48 bits) positions,
//    velocities, accelerations and element forces until the relative residual
//    first drops below lead_tol. Random fiber networks are not isostatic and
//    can pass bifurcation points (Section II); which equilibrium the
//    relaxation settles into is decided in this transient and is sensitive to
//    force errors far below FP32 rounding;
//  * FP32 phase: each element force is an exact increment about a reference
//    state x_ref,
//        t(d_ref + dd) = t(d_ref) + q_ref dd + dq (d_ref + dd),
//        q = N/l = EA (1/L - 1/l),  dq = EA h / (l l_ref (l + l_ref)),
//        h = l^2 - l_ref^2 = 2 d_ref.dd + dd.dd,
//    so every FP32 operation acts on small quantities; the nodal sums of
//    t(d_ref) (g_ref) are evaluated in double-float every rebase_every
//    iterations, when the FP32 increment du is folded into the double-float
//    displacement. Velocity and increment updates are FP32;
//  * the residual norm is summed per warp in FP32 (squares, no cancellation)
//    and across warps and CTAs in double-float; the convergence threshold
//    (tol f_ref)^2 is formed in FP64 and compared in double-float; the
//    stress sum is FP64. FP64 instructions stay out of the iteration loop:
//    GB300 issues them at roughly 1/70 of the FP32 rate.
//
// Synchronisation. The FP32 phase keeps two increment buffers (ping-pong), so
// one cluster barrier per iteration suffices: iteration n writes buffer n&1,
// the barrier publishes it, and the residual of iteration n-1 is tested right
// after that barrier (its state, buffer (n-1)&1, is still intact).
#include <cooperative_groups.h>

#include "df64.cuh"
#include "dr_device.cuh"

namespace cg = cooperative_groups;

namespace fe2 {

namespace {

constexpr int kMaxWarps = 16;  // blocks of at most 512 threads

struct MixedShared {
    float red[2][kMaxParts][kMaxWarps];   // per-warp residual partials of every CTA
    float kred[2][kMaxParts][kMaxWarps];  // kinetic-energy partials
    double sig[kMaxParts][9];             // stress partials, read by rank 0
    double wsum[kMaxWarps][9];            // per-warp stress partials
    float4 *P[kMaxParts];                 // every CTA's x_ref / position-hi array
    float4 *Q[2][kMaxParts];              // every CTA's increment / position-lo arrays
    float *redp[kMaxParts];               // every CTA's red
    float *kredp[kMaxParts];              // every CTA's kred
    double *sigp;                         // rank 0's sig
    int item;
};

struct Part {
    int me, C;
    int f0, nfr;   // own free nodes: RVE-local [f0, f0 + nfr)
    int g0, nfx;   // own fixed nodes: RVE-local n_free + [g0, g0 + nfx)
    int nf;        // RVE free count
    __device__ int gidx(int k) const { return k < nfr ? f0 + k : nf + g0 + (k - nfr); }
    __device__ int m() const { return nfr + nfx; }
};

// Double-float total of the cluster's per-warp partials (buffer `buf`),
// computed warp-parallel on the FP32 pipes: lane l adds entries l, l+32, ...
// and a butterfly of double-float additions finishes the sum. The order is
// fixed, so every warp of every CTA obtains the same bits. GB300 issues FP64
// at a small fraction of its FP32 rate, which would make an FP64 reduction by
// every thread cost more than the iteration itself.
__device__ __forceinline__ df cluster_total(const float (*red)[kMaxParts][kMaxWarps], int buf, int C) {
    const int nw = (blockDim.x + 31) >> 5;
    const int total = C * nw;
    const int lane = threadIdx.x & 31;
    df acc = df_from(0.f);
    for (int j = lane; j < total; j += 32) acc = df_add_f(acc, red[buf][j / nw][j % nw]);
    for (int o = 16; o > 0; o >>= 1) {
        const df other = {__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)};
        acc = df_add(acc, other);
    }
    return acc;
}

// a <= b for double-float values.
__device__ __forceinline__ bool df_le(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

// Publish this thread's FP32 partials (warp-reduced) into every CTA's buffer.
__device__ __forceinline__ void publish(MixedShared &sh, const Part &pt, float v, float kv, bool want_k,
                                        int buf) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (want_k)
        for (int o = 16; o > 0; o >>= 1) kv += __shfl_xor_sync(0xffffffffu, kv, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < pt.C) {
        sh.redp[lane][(buf * kMaxParts + pt.me) * kMaxWarps + warp] = v;
        if (want_k) sh.kredp[lane][(buf * kMaxParts + pt.me) * kMaxWarps + warp] = kv;
    }
}

// Double-float internal force on own node k (Algorithm 1, getInternalForces),
// gathered over its CSR row: g = sum_j EA (1/L - 1/l) (x_j - x_i).
__device__ __forceinline__ void gather_df(const DevMesh &M, const RveDesc &R, const int32_t *rowptr,
                                          const MixedShared &sh, const Part &pt, int k,
                                          const float4 *Pl, const float4 *Ql, int qbuf, df &g0,
                                          df &g1, df &g2) {
    const int gi = pt.gidx(k);
    const float4 pi = Pl[k], qi = Ql[k];
    const df xi0 = {pi.x, qi.x}, xi1 = {pi.y, qi.y}, xi2 = {pi.z, qi.z};
    g0 = df_from(0.f); g1 = df_from(0.f); g2 = df_from(0.f);
    const int beg = rowptr[gi], end = rowptr[gi + 1];
    for (int e = beg; e < end; ++e) {
        const int64_t kk = R.csr0 + e;
        const int cp = M.col_part[kk];
        const int r = cp >> 16, loc = cp & 0xffff;
        const float4 pj = r == pt.me ? Pl[loc] : sh.P[r][loc];
        const float4 qj = r == pt.me ? Ql[loc] : sh.Q[qbuf][r][loc];
        const df d0 = df_sub({pj.x, qj.x}, xi0);
        const df d1 = df_sub({pj.y, qj.y}, xi1);
        const df d2 = df_sub({pj.z, qj.z}, xi2);
        const df l2 = df_add(df_add(df_sqr(d0), df_sqr(d1)), df_sqr(d2));
        const df rl = df_rsqrt(l2);
        const float2 eh = M.eaf[kk], el = M.eaf_lo[kk];
        const df q = df_mul({eh.x, el.x}, df_sub({eh.y, el.y}, rl));
        g0 = df_add(g0, df_mul(q, d0));
        g1 = df_add(g1, df_mul(q, d1));
        g2 = df_add(g2, df_mul(q, d2));
    }
}

__device__ void solve_rve_mixed(cg::cluster_group &cl, MixedShared &sh, const DevMesh &M,
                                const DevState &S, const DevResults &O, const SolveParams &P,
                                int p, float4 *Pl, float4 *Q0, float4 *Q1, int &rb) {
    const RveDesc R = M.rve[p];
    const int n = R.n_nodes, nf = R.n_free;
    const int64_t n0 = R.node0, b3 = 3 * n0;
    const int32_t *rowptr = M.rowptr + R.rp0;
    const int32_t *po = M.part_off + (int64_t)p * 2 * (kMaxParts + 1);
    Part pt;
    pt.me = (int)cl.block_rank();
    pt.C = (int)cl.num_blocks();
    pt.nf = nf;
    pt.f0 = po[pt.me];
    pt.nfr = po[pt.me + 1] - pt.f0;
    pt.g0 = po[kMaxParts + 1 + pt.me];
    pt.nfx = po[kMaxParts + 1 + pt.me + 1] - pt.g0;
    const int m = pt.m();
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = P.F[9 * (int64_t)p + k];
    // per-RVE [3][n] blocks
    const float *Xh = M.Xh + b3, *Xl = M.Xl + b3;
    float *uh = S.uh + b3, *ul = S.ul + b3, *vh = S.vh + b3, *vl = S.vl + b3;
    float *ah = S.ah + b3, *al = S.al + b3, *fg = S.fg + b3;
    const float *imh = M.imh + n0, *iml = M.iml + n0;
    double *xg = S.xg + b3;
    const bool want_k = P.want_ke != 0;
    float4 *Qb[2] = {Q0, Q1};

    // ---- setup: affine positions, f_ref, initial state (Algorithm 1) ----
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int i = pt.gidx(k);
        const double X[3] = {M.X0[n0 + i], M.X1[n0 + i], M.X2[n0 + i]};
        double xa[3];
        for (int r = 0; r < 3; ++r)
            xa[r] = dadd(dadd(dmul(F[3 * r], X[0]), dmul(F[3 * r + 1], X[1])), dmul(F[3 * r + 2], X[2]));
        const df a0 = df_from_double(xa[0]), a1 = df_from_double(xa[1]), a2 = df_from_double(xa[2]);
        Pl[k] = make_float4(a0.hi, a1.hi, a2.hi, 0.f);
        Q0[k] = make_float4(a0.lo, a1.lo, a2.lo, 0.f);
        const bool fixed = k >= pt.nfr;
        const double *uw[3] = {S.u0 + n0, S.u1 + n0, S.u2 + n0};
        for (int r = 0; r < 3; ++r) {
            const double uaff = dsub(xa[r], X[r]);
            double u;
            if (fixed || P.init == 1) u = uaff;
            else if (P.init == 2) u = uw[r][i];
            else u = 0.0;
            const df ud = df_from_double(u);
            uh[r * n + i] = ud.hi;
            ul[r * n + i] = ud.lo;
        }
    }
    cl.sync();
    float acc = 0.f;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        df g0, g1, g2;
        gather_df(M, R, rowptr, sh, pt, k, Pl, Q0, 0, g0, g1, g2);
        acc += g0.hi * g0.hi + g1.hi * g1.hi + g2.hi * g2.hi;
    }
    publish(sh, pt, acc, 0.f, false, rb);
    cl.sync();
    const double f_aff = sqrt(df_to_double(cluster_total(sh.red, rb, pt.C)));
    rb ^= 1;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int i = pt.gidx(k);
        df x[3];
        for (int r = 0; r < 3; ++r)
            x[r] = df_add({Xh[r * n + i], Xl[r * n + i]}, {uh[r * n + i], ul[r * n + i]});
        Pl[k] = make_float4(x[0].hi, x[1].hi, x[2].hi, 0.f);
        Q0[k] = make_float4(x[0].lo, x[1].lo, x[2].lo, 0.f);
    }
    cl.sync();
    acc = 0.f;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        df g[3];
        gather_df(M, R, rowptr, sh, pt, k, Pl, Q0, 0, g[0], g[1], g[2]);
        acc += g[0].hi * g[0].hi + g[1].hi * g[1].hi + g[2].hi * g[2].hi;
        if (k < pt.nfr) {
            const int i = pt.gidx(k);
            const df im = {imh[i], iml[i]};
            for (int r = 0; r < 3; ++r) {
                const df a = df_mul(g[r], im);
                ah[r * n + i] = a.hi; al[r * n + i] = a.lo;
                vh[r * n + i] = 0.f; vl[r * n + i] = 0.f;
                fg[r * n + i] = g[r].hi;
            }
        }
    }
    publish(sh, pt, acc, 0.f, false, rb);
    cl.sync();
    const double f0 = sqrt(df_to_double(cluster_total(sh.red, rb, pt.C)));
    rb ^= 1;
    const double f_ref = f_aff > f0 ? f_aff : f0;
    // convergence and lead tests compare squared norms in double-float
    const df thresh2 = df_from_double(dmul(dmul(P.tol, f_ref), dmul(P.tol, f_ref)));
    const df lead2 = df_from_double(dmul(dmul(P.lead_tol, f_ref), dmul(P.lead_tol, f_ref)));

    const double dt64 = dmul(P.alpha, R.dtc);
    const df dt = df_from_double(dt64), hdt = df_from_double(dmul(0.5, dt64));
    const df cdf = df_from_double(R.c);
    const float dtf = dt.hi, hdtf = hdt.hi, cf = cdf.hi;
    const int K = P.rebase_every > 0 ? P.rebase_every : 512;

    int64_t it = 0, lead = 0;
    int status = RVE_MAXITER;
    df r2 = df_from(0.f), k2 = df_from(0.f);
    bool done = false;
    int fin = -1;  // increment buffer holding the final state (FP32 phase), -1: none

    // ---- lead phase: double-float ----
    for (;;) {
        for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
            const int i = pt.f0 + k;
            df x[3];
            for (int c = 0; c < 3; ++c) {
                df v = {vh[c * n + i], vl[c * n + i]};
                const df a = {ah[c * n + i], al[c * n + i]};
                v = df_add(v, df_mul(hdt, a));
                df u = {uh[c * n + i], ul[c * n + i]};
                u = df_add(u, df_mul(dt, v));
                vh[c * n + i] = v.hi; vl[c * n + i] = v.lo;
                uh[c * n + i] = u.hi; ul[c * n + i] = u.lo;
                x[c] = df_add({Xh[c * n + i], Xl[c * n + i]}, u);
            }
            Pl[k] = make_float4(x[0].hi, x[1].hi, x[2].hi, 0.f);
            Q0[k] = make_float4(x[0].lo, x[1].lo, x[2].lo, 0.f);
        }
        cl.sync();
        float rs = 0.f, kes = 0.f;
        for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
            const int i = pt.f0 + k;
            df g[3];
            gather_df(M, R, rowptr, sh, pt, k, Pl, Q0, 0, g[0], g[1], g[2]);
            const df im = {imh[i], iml[i]};
            float vv = 0.f;
            for (int c = 0; c < 3; ++c) {
                df v = {vh[c * n + i], vl[c * n + i]};
                const df a = df_sub(df_mul(g[c], im), df_mul(cdf, v));
                v = df_add(v, df_mul(hdt, a));
                ah[c * n + i] = a.hi; al[c * n + i] = a.lo;
                vh[c * n + i] = v.hi; vl[c * n + i] = v.lo;
                fg[c * n + i] = g[c].hi;
                rs += g[c].hi * g[c].hi;
                vv += v.hi * v.hi;
            }
            if (want_k) kes += 0.5f * vv / imh[i];
        }
        publish(sh, pt, rs, kes, want_k, rb);
        cl.sync();
        r2 = cluster_total(sh.red, rb, pt.C);
        if (want_k) k2 = cluster_total(sh.kred, rb, pt.C);
        rb ^= 1;
        ++it;
        if (!isfinite(r2.hi)) { status = RVE_NAN; done = true; break; }
        if (df_le(r2, thresh2)) { status = RVE_OK; done = true; break; }
        if (it >= P.max_iter) { status = RVE_MAXITER; done = true; break; }
        if (P.lead_iters >= 0 ? it >= P.lead_iters : df_le(r2, lead2)) break;
    }
    lead = it;

    // ---- FP32 phase: increments about a double-float reference ----
    if (!done) {
        // x_ref = current positions (Pl holds their FP32 rounding), g_ref = fg,
        // increments zero. Remote reads of Q0 ended at the last barrier.
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            Q0[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            Q1[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        int b = 0, since = 0, rbp = 0;
        bool pending = false;
        for (;;) {
            // partial velocity update; displacement increment into buffer b
            {
                const float4 *prev = Qb[b ^ 1];
                float4 *cur = Qb[b];
                for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
                    const int i = pt.f0 + k;
                    const float w0 = vh[i] + hdtf * ah[i];
                    const float w1 = vh[n + i] + hdtf * ah[n + i];
                    const float w2 = vh[2 * n + i] + hdtf * ah[2 * n + i];
                    vh[i] = w0; vh[n + i] = w1; vh[2 * n + i] = w2;
                    const float4 d = prev[k];
                    cur[k] = make_float4(d.x + dtf * w0, d.y + dtf * w1, d.z + dtf * w2, 0.f);
                }
            }
            cl.sync();
            if (pending) {
                // residual of the previous iteration (its state is buffer b^1)
                r2 = cluster_total(sh.red, rbp, pt.C);
                if (want_k) k2 = cluster_total(sh.kred, rbp, pt.C);
                if (!isfinite(r2.hi)) { status = RVE_NAN; fin = b ^ 1; break; }
                if (df_le(r2, thresh2)) { status = RVE_OK; fin = b ^ 1; break; }
                if (it >= P.max_iter) { status = RVE_MAXITER; fin = b ^ 1; break; }
            }
            float4 *cur = Qb[b];
            float rs = 0.f, kes = 0.f;
            if (since >= K) {
                // Rebase: fold the increment into the double-float displacement and
                // stage double-float positions (hi in Pl, lo in buffer b).
                for (int k = threadIdx.x; k < m; k += blockDim.x) {
                    const int i = pt.gidx(k);
                    const float4 d = cur[k];
                    const float dd[3] = {d.x, d.y, d.z};
                    df x[3];
                    for (int c = 0; c < 3; ++c) {
                        df u = {uh[c * n + i], ul[c * n + i]};
                        if (k < pt.nfr) {
                            u = df_add_f(u, dd[c]);
                            uh[c * n + i] = u.hi; ul[c * n + i] = u.lo;
                        }
                        x[c] = df_add({Xh[c * n + i], Xl[c * n + i]}, u);
                    }
                    Pl[k] = make_float4(x[0].hi, x[1].hi, x[2].hi, 0.f);
                    cur[k] = make_float4(x[0].lo, x[1].lo, x[2].lo, 0.f);
                }
                cl.sync();
                for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
                    const int i = pt.f0 + k;
                    df g[3];
                    gather_df(M, R, rowptr, sh, pt, k, Pl, cur, b, g[0], g[1], g[2]);
                    fg[i] = g[0].hi; fg[n + i] = g[1].hi; fg[2 * n + i] = g[2].hi;
                }
                cl.sync();
                for (int k = threadIdx.x; k < m; k += blockDim.x) cur[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                // accelerations and velocities from the reference force
                for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
                    const int i = pt.f0 + k;
                    const float im = imh[i];
                    float vv = 0.f;
                    for (int c = 0; c < 3; ++c) {
                        const float g = fg[c * n + i];
                        float w = vh[c * n + i];
                        const float a = g * im - cf * w;
                        w += hdtf * a;
                        ah[c * n + i] = a;
                        vh[c * n + i] = w;
                        rs += g * g;
                        vv += w * w;
                    }
                    if (want_k) kes += 0.5f * vv / im;
                }
                since = 0;
            } else {
                for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
                    const int i = pt.f0 + k;
                    const float4 pi = Pl[k], qi = cur[k];
                    float g0 = fg[i], g1 = fg[n + i], g2 = fg[2 * n + i];
                    const int beg = rowptr[i], end = rowptr[i + 1];
                    for (int e = beg; e < end; ++e) {
                        const int64_t kk = R.csr0 + e;
                        const int cp = M.col_part[kk];
                        const int rr = cp >> 16, loc = cp & 0xffff;
                        const float2 ei = M.eaf[kk];
                        const float4 pj = rr == pt.me ? Pl[loc] : sh.P[rr][loc];
                        const float4 qj = rr == pt.me ? cur[loc] : sh.Q[b][rr][loc];
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
                    const float im = imh[i];
                    float w0 = vh[i], w1 = vh[n + i], w2 = vh[2 * n + i];
                    const float a0 = g0 * im - cf * w0;
                    const float a1 = g1 * im - cf * w1;
                    const float a2 = g2 * im - cf * w2;
                    w0 += hdtf * a0; w1 += hdtf * a1; w2 += hdtf * a2;
                    ah[i] = a0; ah[n + i] = a1; ah[2 * n + i] = a2;
                    vh[i] = w0; vh[n + i] = w1; vh[2 * n + i] = w2;
                    rs += g0 * g0 + g1 * g1 + g2 * g2;
                    if (want_k) kes += 0.5f * (w0 * w0 + w1 * w1 + w2 * w2) / im;
                }
            }
            // publish this iteration's partials; tested after the next barrier
            publish(sh, pt, rs, kes, want_k, rb);
            rbp = rb;
            rb ^= 1;
            pending = true;
            ++it;
            ++since;
            b ^= 1;
        }
    }

    // ---- final displacement (FP64 output) and positions for the stress ----
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int i = pt.gidx(k);
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
        if (fin >= 0 && k < pt.nfr) d = Qb[fin][k];
        const float dd[3] = {d.x, d.y, d.z};
        double *uo[3] = {S.u0 + n0, S.u1 + n0, S.u2 + n0};
        const double *Xd[3] = {M.X0 + n0, M.X1 + n0, M.X2 + n0};
        for (int c = 0; c < 3; ++c) {
            df u = {uh[c * n + i], ul[c * n + i]};
            if (fin >= 0 && k < pt.nfr) u = df_add_f(u, dd[c]);
            const double ud = df_to_double(u);
            uo[c][i] = ud;
            xg[c * n + i] = dadd(Xd[c][i], ud);
        }
    }
    cl.sync();
    // stress: elements split across the cluster, partials reduced on rank 0
    double s[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) s[k] = 0.0;
    {
        const double *x0 = xg, *x1 = xg + n, *x2 = xg + 2 * n;
        for (int e = pt.me * blockDim.x + threadIdx.x; e < R.n_elems; e += pt.C * blockDim.x) {
            const int64_t ee = R.elem0 + e;
            const int a = M.el_a[ee], bb = M.el_b[ee];
            double d[3] = {dsub(x0[bb], x0[a]), dsub(x1[bb], x1[a]), dsub(x2[bb], x2[a])};
            const double l = dsqrt(dadd(dadd(dmul(d[0], d[0]), dmul(d[1], d[1])), dmul(d[2], d[2])));
            const double q = ddiv(dmul(M.el_EA[ee], dsub(ddiv(l, M.el_L[ee]), 1.0)), l);
#pragma unroll
            for (int rr = 0; rr < 3; ++rr)
#pragma unroll
                for (int c = 0; c < 3; ++c) s[3 * rr + c] = dadd(s[3 * rr + c], dmul(dmul(q, d[rr]), d[c]));
        }
    }
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double v = s[k];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sh.wsum[warp][k] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double t = 0.0;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += sh.wsum[w][threadIdx.x];
        sh.sigp[pt.me * 9 + threadIdx.x] = t;
    }
    cl.sync();
    if (pt.me == 0 && threadIdx.x < 9) {
        double t = 0.0;
        for (int q = 0; q < pt.C; ++q) t += sh.sig[q][threadIdx.x];
        O.sigma[9 * (int64_t)p + threadIdx.x] = ddiv(t, dmul(det3(F), R.V0));
    }
    if (pt.me == 0 && threadIdx.x == 0) {
        const double r = sqrt(df_to_double(r2));
        O.iters[p] = it;
        O.rel_res[p] = f_ref > 0.0 ? r / f_ref : (r > 0.0 ? INFINITY : 0.0);
        O.status[p] = status;
        O.f_ref[p] = f_ref;
        O.ke[p] = want_k ? df_to_double(k2) : 0.0;
        O.lead[p] = lead;
    }
    cl.sync();
}

}  // namespace

__global__ void __launch_bounds__(512) dr_mixed_kernel(DevMesh M, DevState S, DevResults O,
                                                       SolveParams P, int part_cap) {
    extern __shared__ __align__(16) float4 dsm[];
    __shared__ MixedShared sh;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    float4 *Pl = dsm, *Q0 = dsm + part_cap, *Q1 = dsm + 2 * part_cap;
    if ((int)threadIdx.x < C) {
        const int r = threadIdx.x;
        sh.P[r] = cl.map_shared_rank(Pl, r);
        sh.Q[0][r] = cl.map_shared_rank(Q0, r);
        sh.Q[1][r] = cl.map_shared_rank(Q1, r);
        sh.redp[r] = cl.map_shared_rank(&sh.red[0][0][0], r);
        sh.kredp[r] = cl.map_shared_rank(&sh.kred[0][0][0], r);
    }
    if (threadIdx.x == 0) sh.sigp = cl.map_shared_rank(&sh.sig[0][0], 0);
    int rb = 0;
    for (;;) {
        if (cl.block_rank() == 0 && threadIdx.x == 0) sh.item = atomicAdd(P.counter, 1);
        cl.sync();
        const int item = *cl.map_shared_rank(&sh.item, 0);
        cl.sync();
        if (item >= P.queue_len) return;
        solve_rve_mixed(cl, sh, M, S, O, P, P.queue[item], Pl, Q0, Q1, rb);
    }
}

namespace {
cudaLaunchConfig_t mixed_config(int clusters, int parts, int block, size_t smem,
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
}  // namespace

int launch_dr_mixed(const DevMesh &m, const DevState &s, const DevResults &r, const SolveParams &p,
                    int clusters, int parts, int block, size_t smem, void *stream) {
    cudaFuncSetAttribute(dr_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(dr_mixed_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg =
        mixed_config(clusters, parts, block, smem, attr, static_cast<cudaStream_t>(stream));
    const int part_cap = (int)(smem / (3 * sizeof(float4)));
    cudaError_t e = cudaLaunchKernelEx(&cfg, dr_mixed_kernel, m, s, r, p, part_cap);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaGetLastError();
}

int occupancy_dr_mixed(int parts, int block, size_t smem) {
    cudaFuncSetAttribute(dr_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(dr_mixed_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = mixed_config(parts * 64, parts, block, smem, attr, nullptr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, dr_mixed_kernel, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace fe2
