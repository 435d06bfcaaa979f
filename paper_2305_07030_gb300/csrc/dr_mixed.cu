// Mixed-precision dynamic relaxation (Algorithm 1) for a batch of RVEs: one
// thread-block cluster per RVE, three persistent launches per size class (the
// double-float lead, the FP32 phase, the double-float resume of stalled RVEs).
//
// Layout. The RVE is split spatially into `parts` pieces, one per CTA of the
// cluster; a CTA stages the state of its own nodes in its shared memory and
// reads neighbours owned by other CTAs through distributed shared memory. The
// paper used one thread team per sub-problem (Section III); a cluster lets one
// sub-problem span several SMs.
//
// Precision. All arithmetic of the iterations runs on the FP32 pipes (GB300
// issues FP64 at roughly 1/70 of the FP32 rate):
//  * lead kernel: double-float (hi + lo FP32 pairs, ~48 bits) displacement,
//    velocity, acceleration and element forces until the relative residual
//    first drops below lead_tol. Random fiber networks are not isostatic and
//    can pass bifurcation points (Section II); which equilibrium the
//    relaxation settles into is decided in this transient and is sensitive to
//    force errors far below FP32 rounding. Element forces are evaluated in
//    displacement form, d = D + (u_j - u_i) with D = X_j - X_i, and
//    N/l = EA h / (L l (l + L)), h = l^2 - L^2 = (u_j - u_i).(D + d), which
//    has no cancellation, so the double-float strain is accurate to ~1e-14;
//  * FP32 kernel: each element force is an exact increment about a reference
//    state x_ref,
//        t(d_ref + dd) = t(d_ref) + q_ref dd + dq (d_ref + dd),
//        q = N/l = EA (1/L - 1/l),  dq = EA h / (l l_ref (l + l_ref)),
//        h = l^2 - l_ref^2 = 2 d_ref.dd + dd.dd,
//    so every FP32 operation acts on small quantities; the nodal sums of
//    t(d_ref) (g_ref) are evaluated in double-float every rebase_every
//    iterations, when the FP32 increment du is folded into the double-float
//    displacement. Velocity and increment updates are FP32;
//  * the residual norm is summed per warp in FP32 (squares, no cancellation)
//    and across warps and CTAs in double-float; the threshold (tol f_ref)^2 is
//    formed in FP64 once per RVE; the stress sum is FP64.
//
// Synchronisation of the FP32 kernel. One cluster barrier per iteration.
// Five displacement-increment buffers rotate. Each node's owner thread
// computes the next iteration's increment right after the node's velocity
// update, so an iteration begins at the barrier. Between the barrier's arrive
// and wait, every warp publishes its residual partial of the previous
// evaluation to its own CTA, and one warp per CTA totals evaluation n-3 across
// the cluster (DSMEM reads) and leaves a verdict. All warps read the verdict
// after the next barrier. If the test succeeded, they finish with the state of
// the tested evaluation, whose buffer is still intact.
//
// The element forces of the FP32 kernel and of the lead come from a
// shared-memory element table. Each element with an end among a CTA's free
// nodes is evaluated once per iteration, spread evenly over the threads. Each
// node then sums the +- results of its CSR row in row order. The two ends see
// exactly opposite values, so this equals the per-direction evaluation.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "df64.cuh"
#include "dr_device.cuh"

namespace cg = cooperative_groups;

namespace fe2 {

namespace {

constexpr int kMaxWarps = 16;  // blocks of at most 512 threads
constexpr int kLeadBufs = 3;   // lead kernel: rotating partial buffers
constexpr int kBufs = 5;       // FP32 kernel: rotating increment / partial buffers
// FP32 kernel shared memory per node with the element table: reference
// position, five increment buffers (float4 each), velocity + a.x (float4),
// a.yz (float2). Without the table, velocity and acceleration live in global
// memory and a node takes the first six float4 only.
constexpr size_t kFp32NodeBytes = (1 + kBufs + 1) * sizeof(float4) + sizeof(float2);
constexpr size_t kFp32PlainNodeBytes = (1 + kBufs) * sizeof(float4);
// Lead kernel shared memory per node without the element table: one
// double-float displacement (hi, lo float4); with the table, two of them.
constexpr size_t kLeadPlainNodeBytes = 2 * sizeof(float4);
__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Convergence verdict on one evaluation (FP32 kernel): code -1 = go on, else
// the RVE status; the double-float squared residual and kinetic energy.
struct Verdict {
    int code;
    float r2h, r2l, k2h, k2l;
};

struct MixedShared {
    // lead kernel: per-warp residual partials of every CTA, dense: entry
    // (rank * warps + warp)
    float red[kLeadBufs][kMaxParts * kMaxWarps];
    float kred[kLeadBufs][kMaxParts * kMaxWarps]; // kinetic-energy partials
    // FP32 kernel: this CTA's per-warp partials (residual, kinetic energy)
    float own[kBufs][2][kMaxWarps];
    Verdict vd[kBufs];                        // verdicts of the testing warp
    float *ownp[kMaxParts];                   // every CTA's own
    double sig[kMaxParts][9];                 // stress partials, read by rank 0
    double wsum[kMaxWarps][9];                // per-warp stress partials
    float4 *P[kMaxParts];                     // every CTA's position array
    float4 *Q[kBufs][kMaxParts];              // every CTA's increment / low-part arrays
    float *redp[kMaxParts];                   // every CTA's red
    float *kredp[kMaxParts];                  // every CTA's kred
    double *sigp;                             // rank 0's sig
    int item;
    // FP32 kernel stall tracker (testing warp): the squared residual that the
    // next ones must reach a quarter of, and the evaluation that set it
    float st_h, st_l;
    long long st_e;
    int elems;                                // FP32 kernel: elements of this CTA's part
    int slots;                                // FP32 kernel: row slots of this CTA's part
};

struct Part {
    int me, C;
    int f0, nfr;   // own free nodes: RVE-local [f0, f0 + nfr)
    int g0, nfx;   // own fixed nodes: RVE-local n_free + [g0, g0 + nfx)
    int nf;        // RVE free count
    __device__ int gidx(int k) const { return k < nfr ? f0 + k : nf + g0 + (k - nfr); }
    __device__ int m() const { return nfr + nfx; }
};

__device__ __forceinline__ Part make_part(const DevMesh &M, const RveDesc &R, int p, int me, int C) {
    const int32_t *po = M.part_off + (int64_t)p * 2 * (kMaxParts + 1);
    Part pt;
    pt.me = me;
    pt.C = C;
    pt.nf = R.n_free;
    pt.f0 = po[me];
    pt.nfr = po[me + 1] - pt.f0;
    pt.g0 = po[kMaxParts + 1 + me];
    pt.nfx = po[kMaxParts + 1 + me + 1] - pt.g0;
    return pt;
}

__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Double-float total of the cluster's per-warp partials (buffer `buf`),
// computed warp-parallel on the FP32 pipes: lane l adds entries l, l+32, ...
// and a butterfly of double-float additions finishes the sum. The order is
// fixed, so every warp of every CTA obtains the same bits. GB300 issues FP64
// at a small fraction of its FP32 rate, which would make an FP64 reduction by
// every thread cost more than the iteration itself.
__device__ __forceinline__ df cluster_total(const float (*red)[kMaxParts * kMaxWarps], int buf, int C) {
    const int total = C * (int)(blockDim.x >> 5);
    const int lane = threadIdx.x & 31;
    df acc = df_from(0.f);
    for (int j = lane; j < total; j += 32) acc = df_add_f(acc, red[buf][j]);
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
    const int slot = buf * (kMaxParts * kMaxWarps) + pt.me * (int)(blockDim.x >> 5) + warp;
    if (lane < pt.C) {
        sh.redp[lane][slot] = v;
        if (want_k) sh.kredp[lane][slot] = kv;
    }
}

// Combine double-float partial sums over groups of L consecutive lanes (every
// lane of the warp must call this).
__device__ __forceinline__ void df_group_sum(df &g0, df &g1, df &g2, int L) {
    for (int o = 1; o < L; o <<= 1) {
        const df a0 = {__shfl_xor_sync(0xffffffffu, g0.hi, o), __shfl_xor_sync(0xffffffffu, g0.lo, o)};
        const df a1 = {__shfl_xor_sync(0xffffffffu, g1.hi, o), __shfl_xor_sync(0xffffffffu, g1.lo, o)};
        const df a2 = {__shfl_xor_sync(0xffffffffu, g2.hi, o), __shfl_xor_sync(0xffffffffu, g2.lo, o)};
        g0 = df_add(g0, a0);
        g1 = df_add(g1, a1);
        g2 = df_add(g2, a2);
    }
}

// Double-float internal force on own node k (Algorithm 1, getInternalForces)
// in displacement form; the node's and its neighbours' displacements are
// staged as (hi, lo) in (Pl, Ql) and the other CTAs' copies (Q buffer qbuf).
__device__ __forceinline__ void gather_df(const DevMesh &M, const RveDesc &R, const int32_t *rowptr,
                                          const MixedShared &sh, const Part &pt, int k,
                                          const float4 *Pl, const float4 *Ql, int qbuf, df &g0,
                                          df &g1, df &g2, int sub = 0, int L = 1) {
    const int gi = pt.gidx(k);
    const float4 pi = Pl[k], qi = Ql[k];
    const df ui0 = {pi.x, qi.x}, ui1 = {pi.y, qi.y}, ui2 = {pi.z, qi.z};
    g0 = df_from(0.f); g1 = df_from(0.f); g2 = df_from(0.f);
    const int beg = rowptr[gi], end = rowptr[gi + 1];
    // lane `sub` of L takes edges sub, sub+L, ... (the caller combines the lanes)
    for (int e = beg + sub; e < end; e += L) {
        const int64_t kk = R.csr0 + e;
        const int cp = M.col_part[kk];
        const int r = cp >> 16, loc = cp & 0xffff;
        const float4 pj = r == pt.me ? Pl[loc] : sh.P[r][loc];
        const float4 qj = r == pt.me ? Ql[loc] : sh.Q[qbuf][r][loc];
        const float4 Dh = M.dh[kk], Dl = M.dl[kk];
        // relative displacement and current element vector
        const df e0 = df_sub({pj.x, qj.x}, ui0), e1 = df_sub({pj.y, qj.y}, ui1),
                 e2 = df_sub({pj.z, qj.z}, ui2);
        const df D0 = {Dh.x, Dl.x}, D1 = {Dh.y, Dl.y}, D2 = {Dh.z, Dl.z}, L = {Dh.w, Dl.w};
        const df d0 = df_add(D0, e0), d1 = df_add(D1, e1), d2 = df_add(D2, e2);
        // h = l^2 - L^2 = e.(D + d)
        const df h = df_add(df_add(df_mul(e0, df_add(D0, d0)), df_mul(e1, df_add(D1, d1))),
                            df_mul(e2, df_add(D2, d2)));
        const df l2 = df_add(df_sqr(L), h);
        const df rl = df_rsqrt(l2);
        const df l = df_mul(l2, rl);
        const float2 eh = M.eaf[kk], el = M.eaf_lo[kk];
        // N/l = EA (l - L) / (L l) = (EA/L) h / (l (l + L))
        const df kax = df_mul({eh.x, el.x}, {eh.y, el.y});
        const df q = df_mul(df_mul(kax, df_mul(h, rl)), df_rcp(df_add(l, L)));
        g0 = df_add(g0, df_mul(q, d0));
        g1 = df_add(g1, df_mul(q, d1));
        g2 = df_add(g2, df_mul(q, d2));
    }
}

__device__ __forceinline__ void map_remote(cg::cluster_group &cl, MixedShared &sh, float4 *Pl,
                                           float4 *const *Qb, int C) {
    if ((int)threadIdx.x < C) {
        const int r = threadIdx.x;
        sh.P[r] = cl.map_shared_rank(Pl, r);
        for (int b = 0; b < kBufs; ++b) sh.Q[b][r] = cl.map_shared_rank(Qb[b], r);
        sh.redp[r] = cl.map_shared_rank(&sh.red[0][0], r);
        sh.kredp[r] = cl.map_shared_rank(&sh.kred[0][0], r);
        sh.ownp[r] = cl.map_shared_rank(&sh.own[0][0][0], r);
    }
    if (threadIdx.x == 0) sh.sigp = cl.map_shared_rank(&sh.sig[0][0], 0);
}

// Next work item of the cluster (rank 0 pops, everyone reads it).
__device__ __forceinline__ int next_item(cg::cluster_group &cl, MixedShared &sh, int32_t *counter) {
    if (cl.block_rank() == 0 && threadIdx.x == 0) sh.item = atomicAdd(counter, 1);
    cl.sync();
    const int item = *cl.map_shared_rank(&sh.item, 0);
    cl.sync();
    return item;
}

// FP32 increment of one element's force on node i from neighbour j about the
// reference state: t(d_ref + dd) - t(d_ref) + q_ref dd, accumulated into g.
// p* hold FP32 reference positions, q* the FP32 displacement increments;
// ei = (EA, 1/L).
__device__ __forceinline__ void edge_increment(const float4 &pi, const float4 &qi, const float4 &pj,
                                               const float4 &qj, float2 ei, float &g0, float &g1,
                                               float &g2) {
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

// Per-part element tables of the FP32 kernel, in shared memory when they fit
// (STAGE); otherwise every row is re-read from the global CSR each iteration.
//
// Element list: each element with at least one end among this CTA's free
// nodes appears once. An element between two own free nodes belongs to the
// row of its lower local index (end a) and is used with the opposite sign by
// the other row (end b); any other element belongs to the row of its own free
// end a. Element u holds
//   K0 = (r, |r|^2), r = x_ref,b - x_ref,a,
//   K1 = (q_ref, EA, 1/|r|, address of b's increment in buffer 0: shared::cta,
//        or shared::cluster with bit 0 set when b lives in another CTA),
//   EI = shared::cta address of a's increment in buffer 0,
//   TF = the iteration's force increment on a (on b it is -TF, exactly).
// The reference geometry only changes when the reference state moves.
// Node rows are laid out ELL-style in slabs of 32 consecutive own free nodes:
// entry j of node k sits at slot SS[k / 32] + 32 j + k % 32 and holds
// (element << 1 | 1 if the node is end b), so a warp reads 32 consecutive
// slots at every step; the entries keep the CSR row order.
struct Staged {
    float4 *SG;    // per own free node: (g_ref, 1/m)
    float4 *K0;    // per element
    float4 *K1;    // per element
    float4 *TF;    // per element
    uint32_t *EI;  // per element
    uint32_t *NS;  // per slot
    int *SD;       // per own free node: row length
    int *EB;       // per own free node: first element of its row
    int *SS;       // per slab + 1: first slot
    // lead kernel only (K0, K1 then hold the double-float D and L)
    float4 *KA;    // per element
    float4 *TA;    // per element
    float2 *TB;    // per element
    float4 *VH;    // per own free node: (v.hi, a.hi x)
    float4 *VL;    // per own free node: (v.lo, a.lo x)
    float4 *AY;    // per own free node: (a.hi y, a.hi z, a.lo y, a.lo z)
};

// 32-bit shared-memory address of p and its image in cluster CTA `rank`.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_addr(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ float4 ld_cluster(uint32_t a) {
    float4 v;
    asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a));
    return v;
}
__device__ __forceinline__ float4 ld_local(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(a));
    return v;
}

// The FP32 increment of edge_increment with the reference geometry taken from
// an element's K0, K1 (same operations, same order).
__device__ __forceinline__ void edge_increment_slot(const float4 &qi, const float4 &qj, const float4 &k0,
                                                    const float4 &k1, float &g0, float &g1, float &g2) {
    const float r0 = k0.x, r1 = k0.y, r2 = k0.z, lr2 = k0.w;
    const float qref = k1.x, ea = k1.y, ril = k1.z;
    const float e0 = qj.x - qi.x, e1 = qj.y - qi.y, e2 = qj.z - qi.z;
    const float lr = lr2 * ril;
    const float h = 2.f * (r0 * e0 + r1 * e1 + r2 * e2) + (e0 * e0 + e1 * e1 + e2 * e2);
    const float rl = rsqrtf(lr2 + h);
    const float l = (lr2 + h) * rl;
    const float dq = __fdividef(ea * h * rl * ril, l + lr);
    g0 += qref * e0 + dq * (r0 + e0);
    g1 += qref * e1 + dq * (r1 + e1);
    g2 += qref * e2 + dq * (r2 + e2);
}

// Whether CSR entry (rank r, local loc) of own free node k is used with the
// opposite sign: its element belongs to the lower own free end.
__device__ __forceinline__ bool b_end(int r, int loc, int k, const Part &pt) {
    return r == pt.me && loc < pt.nfr && loc < k;
}

// Row lengths and element counts of this CTA's free nodes (first pass), then
// (thread 0) element offsets and slab bases. The caller synchronises the CTA
// before the second part.
__device__ void element_counts(const DevMesh &M, const RveDesc &R, const Part &pt, const int32_t *rowptr,
                               const Staged &st) {
    for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
        const int beg = rowptr[pt.f0 + k], deg = rowptr[pt.f0 + k + 1] - beg;
        int own = 0;
        for (int e = 0; e < deg; ++e) {
            const int cp = M.col_part[R.csr0 + beg + e];
            own += !b_end(cp >> 16, cp & 0xffff, k, pt);
        }
        st.SD[k] = deg;
        st.EB[k] = own;
    }
}
__device__ void element_offsets(MixedShared &sh, const Part &pt, const Staged &st) {
    int base = 0;
    for (int k = 0; k < pt.nfr; ++k) {
        const int c = st.EB[k];
        st.EB[k] = base;
        base += c;
    }
    sh.elems = base;
    int slots = 0, s = 0;
    for (int k0 = 0; k0 < pt.nfr; k0 += 32, ++s) {
        int w = 0;
        for (int k = k0; k < k0 + 32 && k < pt.nfr; ++k) w = max(w, st.SD[k]);
        st.SS[s] = slots;
        slots += 32 * w;
    }
    st.SS[s] = slots;
    sh.slots = slots;
}

// Fill the element table from the current reference positions (every CTA's Pl
// must be final): K0 and K1.xyz always; with `full` also the addresses and the
// node rows.
__device__ void element_setup(const MixedShared &sh, const DevMesh &M, const RveDesc &R, const Part &pt,
                              const int32_t *rowptr, const float4 *Pl, const float4 *Q0,
                              const Staged &st, bool full) {
    for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
        const int beg = rowptr[pt.f0 + k], deg = st.SD[k];
        const float4 pa = Pl[k];
        int u = st.EB[k];
        int slot = st.SS[k >> 5] + (k & 31);
        for (int e = 0; e < deg; ++e, slot += 32) {
            const int64_t kk = R.csr0 + beg + e;
            const int cp = M.col_part[kk];
            const int r = cp >> 16, loc = cp & 0xffff;
            if (b_end(r, loc, k, pt)) {
                if (full) {
                    // the element's index in row loc
                    const int jb = rowptr[pt.f0 + loc], jd = st.SD[loc];
                    int v = st.EB[loc];
                    for (int x = 0; x < jd; ++x) {
                        const int cq = M.col_part[R.csr0 + jb + x];
                        const int rq = cq >> 16, lq = cq & 0xffff;
                        if (rq == pt.me && lq == k) break;
                        v += !b_end(rq, lq, loc, pt);
                    }
                    st.NS[slot] = ((uint32_t)v << 1) | 1u;
                }
                continue;
            }
            const float4 pb = r == pt.me ? Pl[loc] : sh.P[r][loc];
            const float2 ei = M.eaf[kk];
            const float r0 = pb.x - pa.x, r1 = pb.y - pa.y, r2 = pb.z - pa.z;
            const float lr2 = r0 * r0 + r1 * r1 + r2 * r2;
            const float ril = rsqrtf(lr2);
            const float qref = ei.x * (ei.y - ril);
            uint32_t ab;
            if (full) {
                const uint32_t qb = smem_addr(Q0 + loc);
                ab = r == pt.me ? qb : (cluster_addr(qb, (uint32_t)r) | 1u);
                st.EI[u] = smem_addr(Q0 + k);
                st.NS[slot] = (uint32_t)u << 1;
            } else {
                ab = __float_as_uint(st.K1[u].w);
            }
            st.K0[u] = make_float4(r0, r1, r2, lr2);
            st.K1[u] = make_float4(qref, ei.x, ril, __uint_as_float(ab));
            ++u;
        }
    }
}

// Convergence verdict on one evaluation: the double-float total of every
// CTA's per-warp partials (fixed order: rank, then warp), read through
// distributed shared memory.
__device__ __forceinline__ Verdict residual_verdict(const MixedShared &sh, const Part &pt, int buf, int64_t done,
                                         const df &thresh2, bool want_k, int64_t max_iter) {
    const int nw = (int)(blockDim.x >> 5), total = pt.C * nw, lane = threadIdx.x & 31;
    df r2 = df_from(0.f), k2 = df_from(0.f);
    for (int j = lane; j < total; j += 32) {
        const int r = j / nw, w = j - r * nw;
        r2 = df_add_f(r2, sh.ownp[r][(buf * 2 + 0) * kMaxWarps + w]);
        if (want_k) k2 = df_add_f(k2, sh.ownp[r][(buf * 2 + 1) * kMaxWarps + w]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        r2 = df_add(r2, {__shfl_xor_sync(0xffffffffu, r2.hi, o), __shfl_xor_sync(0xffffffffu, r2.lo, o)});
        if (want_k)
            k2 = df_add(k2, {__shfl_xor_sync(0xffffffffu, k2.hi, o), __shfl_xor_sync(0xffffffffu, k2.lo, o)});
    }
    Verdict v;
    v.code = !isfinite(r2.hi) ? RVE_NAN : df_le(r2, thresh2) ? RVE_OK : done >= max_iter ? RVE_MAXITER : -1;
    v.r2h = r2.hi; v.r2l = r2.lo; v.k2h = k2.hi; v.k2l = k2.lo;
    return v;
}

// ---------------------------------------------------------------------------
// lead kernel with the element table (STAGE)
// ---------------------------------------------------------------------------
// The lead's element table: the same element list and node rows as the FP32
// kernel's (element_counts, element_offsets), with per element
//   K0 = (D, L).hi, K1 = (D, L).lo  (D = X_b - X_a, double-float),
//   KA = ((EA/L).hi, (EA/L).lo, shared::cta address of a's displacement in
//        buffer 0, address of b's: shared::cta, or shared::cluster with bit 0
//        set when b lives in another CTA),
//   TA, TB = the iteration's double-float force on a (hi xyz + lo x; lo yz).
// Displacements rotate through two buffers (hi then lo arrays per buffer), so
// one cluster barrier per iteration suffices.
__device__ void lead_elements(const MixedShared &sh, const DevMesh &M, const RveDesc &R, const Part &pt,
                              const int32_t *rowptr, const float4 *U0, const Staged &st) {
    for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
        const int beg = rowptr[pt.f0 + k], deg = st.SD[k];
        int u = st.EB[k];
        int slot = st.SS[k >> 5] + (k & 31);
        for (int e = 0; e < deg; ++e, slot += 32) {
            const int64_t kk = R.csr0 + beg + e;
            const int cp = M.col_part[kk];
            const int r = cp >> 16, loc = cp & 0xffff;
            if (b_end(r, loc, k, pt)) {
                const int jb = rowptr[pt.f0 + loc], jd = st.SD[loc];
                int v = st.EB[loc];
                for (int x = 0; x < jd; ++x) {
                    const int cq = M.col_part[R.csr0 + jb + x];
                    const int rq = cq >> 16, lq = cq & 0xffff;
                    if (rq == pt.me && lq == k) break;
                    v += !b_end(rq, lq, loc, pt);
                }
                st.NS[slot] = ((uint32_t)v << 1) | 1u;
                continue;
            }
            const float2 eh = M.eaf[kk], el = M.eaf_lo[kk];
            const df kax = df_mul({eh.x, el.x}, {eh.y, el.y});
            const uint32_t qb = smem_addr(U0 + loc);
            const uint32_t ab = r == pt.me ? qb : (cluster_addr(qb, (uint32_t)r) | 1u);
            st.K0[u] = M.dh[kk];
            st.K1[u] = M.dl[kk];
            st.KA[u] = make_float4(kax.hi, kax.lo, __uint_as_float(smem_addr(U0 + k)), __uint_as_float(ab));
            st.NS[slot] = (uint32_t)u << 1;
            ++u;
        }
    }
}

__device__ __forceinline__ float4 ld_any(uint32_t a) {
    return (a & 1u) ? ld_cluster(a & ~1u) : ld_local(a);
}

// Double-float element force in displacement form (the operations of
// gather_df) for element u, written to TA/TB.
__device__ __forceinline__ void lead_element_force(const Staged &st, int u, const float4 &pi,
                                                   const float4 &qi, const float4 &pj, const float4 &qj) {
    const float4 Dh = st.K0[u], Dl = st.K1[u];
    const float2 kax = make_float2(st.KA[u].x, st.KA[u].y);
    const df e0 = df_sub({pj.x, qj.x}, {pi.x, qi.x}), e1 = df_sub({pj.y, qj.y}, {pi.y, qi.y}),
             e2 = df_sub({pj.z, qj.z}, {pi.z, qi.z});
    const df D0 = {Dh.x, Dl.x}, D1 = {Dh.y, Dl.y}, D2 = {Dh.z, Dl.z}, L = {Dh.w, Dl.w};
    const df d0 = df_add(D0, e0), d1 = df_add(D1, e1), d2 = df_add(D2, e2);
    const df h = df_add(df_add(df_mul(e0, df_add(D0, d0)), df_mul(e1, df_add(D1, d1))),
                        df_mul(e2, df_add(D2, d2)));
    const df l2 = df_add(df_sqr(L), h);
    const df rl = df_rsqrt(l2);
    const df l = df_mul(l2, rl);
    const df q = df_mul(df_mul({kax.x, kax.y}, df_mul(h, rl)), df_rcp(df_add(l, L)));
    const df t0 = df_mul(q, d0), t1 = df_mul(q, d1), t2 = df_mul(q, d2);
    st.TA[u] = make_float4(t0.hi, t1.hi, t2.hi, t0.lo);
    st.TB[u] = make_float2(t1.lo, t2.lo);
}

// Elements ua and ub (ub < 0: none) of displacement buffer offset toff: all
// loads first, then the two independent chains.
__device__ __forceinline__ void lead_element_pair(const Staged &st, int ua, int ub, uint32_t toff,
                                                  uint32_t lo_off) {
    const float4 ka = st.KA[ua];
    const uint32_t a0 = __float_as_uint(ka.z) + toff, a1 = __float_as_uint(ka.w) + toff;
    const float4 pi = ld_local(a0), qi = ld_local(a0 + lo_off);
    const float4 pj = ld_any(a1), qj = ld_any(a1 + lo_off);
    if (ub >= 0) {
        const float4 kb = st.KA[ub];
        const uint32_t b0 = __float_as_uint(kb.z) + toff, b1 = __float_as_uint(kb.w) + toff;
        const float4 pi2 = ld_local(b0), qi2 = ld_local(b0 + lo_off);
        const float4 pj2 = ld_any(b1), qj2 = ld_any(b1 + lo_off);
        lead_element_force(st, ua, pi, qi, pj, qj);
        lead_element_force(st, ub, pi2, qi2, pj2, qj2);
    } else {
        lead_element_force(st, ua, pi, qi, pj, qj);
    }
}

// Double-float iterations until the relative residual first drops below
// lead_tol (or lead_iters), NaN or max_iter. The residual test of evaluation
// n-2 runs in one testing warp per CTA between the arrive and the wait of
// iteration n; the others read its verdict after the next barrier, and the
// hand-over happens at the end of that iteration, so the handed-over state
// (u, v, a and g_ref of one evaluation) is consistent. The hand-over state's
// own residual is then totalled by every warp.
__device__ void lead_loop_staged(cg::cluster_group &cl, MixedShared &sh, const DevMesh &M,
                                 const DevState &S, const RveDesc &R, const Part &pt,
                                 const SolveParams &P, float4 *U0, const Staged &st, int part_cap,
                                 int elem_cap, int slot_cap, const df &lead2, const df &thresh2,
                                 const df &dt, const df &hdt, const df &cdf, int64_t &it,
                                 int &status, df &r2, df &k2) {
    const int64_t it0 = it;  // evaluations before this call (resume: > 0)
    const int n = R.n_nodes, m = pt.m();
    const int64_t n0 = R.node0, b3 = 3 * n0;
    const int32_t *rowptr = M.rowptr + R.rp0;
    float *uh = S.uh + b3, *ul = S.ul + b3, *vh = S.vh + b3, *vl = S.vl + b3;
    float *ah = S.ah + b3, *al = S.al + b3, *fg = S.fg + b3;
    const float *imh = M.imh + n0, *iml = M.iml + n0;
    const bool want_k = P.want_ke != 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool test_warp = warp == (int)(blockDim.x >> 5) - 1;
    // buffer t: hi at U0 + 2 t part_cap, lo at U0 + (2 t + 1) part_cap
    const uint32_t lo_off = (uint32_t)(sizeof(float4) * part_cap), buf_off = 2 * lo_off;
    // buffer 1 starts as a copy of buffer 0 (the fixed nodes never change)
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        U0[2 * part_cap + k] = U0[k];
        U0[3 * part_cap + k] = U0[part_cap + k];
    }
    element_counts(M, R, pt, rowptr, st);
    __syncthreads();
    if (threadIdx.x == 0) element_offsets(sh, pt, st);
    cl.sync();
    bool over = false;
    for (int r = 0; r < pt.C; ++r)
        over |= *cl.map_shared_rank(&sh.elems, r) > elem_cap || *cl.map_shared_rank(&sh.slots, r) > slot_cap;
    if (over) {  // sized on the host for every part; all CTAs agree
        status = RVE_NAN;
        return;
    }
    lead_elements(sh, M, R, pt, rowptr, U0, st);
    const int n_el = sh.elems;
    // velocity and acceleration of the own free nodes live in shared memory
    // during the loop (owner thread k in every phase)
    for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
        const int i = pt.f0 + k;
        st.VH[k] = make_float4(vh[i], vh[n + i], vh[2 * n + i], ah[i]);
        st.VL[k] = make_float4(vl[i], vl[n + i], vl[2 * n + i], al[i]);
        st.AY[k] = make_float4(ah[n + i], ah[2 * n + i], al[n + i], al[2 * n + i]);
    }
    __syncthreads();

    bool vpend = false;
    for (;;) {
        const int64_t nidx = it + 1;  // this iteration's evaluation
        const int t = (int)(nidx & 1), tp = t ^ 1;
        const int vb = (int)(nidx & 3);
        {
            const float4 *Hp = U0 + 2 * tp * part_cap, *Lp = Hp + part_cap;
            float4 *Hc = U0 + 2 * t * part_cap, *Lc = Hc + part_cap;
            for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
                const float4 ph = Hp[k], pl = Lp[k];
                const float4 vhk = st.VH[k], vlk = st.VL[k], ay = st.AY[k];
                const float uh0[3] = {ph.x, ph.y, ph.z}, ul0[3] = {pl.x, pl.y, pl.z};
                const float v_h[3] = {vhk.x, vhk.y, vhk.z}, v_l[3] = {vlk.x, vlk.y, vlk.z};
                const float a_h[3] = {vhk.w, ay.x, ay.y}, a_l[3] = {vlk.w, ay.z, ay.w};
                df u[3], v[3];
                for (int c = 0; c < 3; ++c) {
                    v[c] = df_add({v_h[c], v_l[c]}, df_mul(hdt, {a_h[c], a_l[c]}));
                    u[c] = df_add({uh0[c], ul0[c]}, df_mul(dt, v[c]));
                }
                st.VH[k] = make_float4(v[0].hi, v[1].hi, v[2].hi, vhk.w);
                st.VL[k] = make_float4(v[0].lo, v[1].lo, v[2].lo, vlk.w);
                Hc[k] = make_float4(u[0].hi, u[1].hi, u[2].hi, 0.f);
                Lc[k] = make_float4(u[0].lo, u[1].lo, u[2].lo, 0.f);
            }
        }
        const bool test_now = nidx >= it0 + 3;  // two evaluations of this call published
        cluster_arrive();
        if (test_now && test_warp) {
            const Verdict v = residual_verdict(sh, pt, (int)((nidx - 2) & 3), 0, lead2, want_k, INT64_MAX);
            if (lane == 0) sh.vd[vb] = v;
        }
        cluster_wait();
        const int code = vpend ? sh.vd[(nidx - 1) & 3].code : -1;
        vpend = test_now;
        // element forces in displacement form (gather_df's operations), two
        // elements per thread in flight
        const uint32_t toff = (uint32_t)t * buf_off;
        const int step = blockDim.x;
        for (int u0 = threadIdx.x; u0 < n_el; u0 += 2 * step) {
            lead_element_pair(st, u0, u0 + step < n_el ? u0 + step : -1, toff, lo_off);
        }
        __syncthreads();
        // node sums in CSR row order, then acceleration and velocity
        float rs = 0.f, kes = 0.f;
        for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
            const int deg = st.SD[k];
            int sl = st.SS[k >> 5] + (k & 31);
            df g[3] = {df_from(0.f), df_from(0.f), df_from(0.f)};
            for (int j = 0; j < deg; ++j, sl += 32) {
                const uint32_t w = st.NS[sl];
                const float4 ta = st.TA[w >> 1];
                const float2 tb = st.TB[w >> 1];
                df f0 = {ta.x, ta.w}, f1 = {ta.y, tb.x}, f2 = {ta.z, tb.y};
                if (w & 1u) {
                    f0 = {-f0.hi, -f0.lo}; f1 = {-f1.hi, -f1.lo}; f2 = {-f2.hi, -f2.lo};
                }
                g[0] = df_add(g[0], f0); g[1] = df_add(g[1], f1); g[2] = df_add(g[2], f2);
            }
            const int i = pt.f0 + k;
            const df im = {imh[i], iml[i]};
            const float4 vhk = st.VH[k], vlk = st.VL[k];
            const float v_h[3] = {vhk.x, vhk.y, vhk.z}, v_l[3] = {vlk.x, vlk.y, vlk.z};
            float vv = 0.f;
            df v[3], a[3];
            for (int c = 0; c < 3; ++c) {
                v[c] = {v_h[c], v_l[c]};
                a[c] = df_sub(df_mul(g[c], im), df_mul(cdf, v[c]));
                v[c] = df_add(v[c], df_mul(hdt, a[c]));
                fg[c * n + i] = g[c].hi;
                rs += g[c].hi * g[c].hi;
                vv += v[c].hi * v[c].hi;
            }
            st.VH[k] = make_float4(v[0].hi, v[1].hi, v[2].hi, a[0].hi);
            st.VL[k] = make_float4(v[0].lo, v[1].lo, v[2].lo, a[0].lo);
            st.AY[k] = make_float4(a[1].hi, a[2].hi, a[1].lo, a[2].lo);
            if (want_k) kes += 0.5f * vv / imh[i];
        }
        for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
        if (want_k)
            for (int o = 16; o > 0; o >>= 1) kes += __shfl_xor_sync(0xffffffffu, kes, o);
        if (lane == 0) {
            sh.own[vb][0][warp] = rs;
            if (want_k) sh.own[vb][1][warp] = kes;
        }
        it = nidx;
        if (code == RVE_NAN) break;
        if (it >= P.max_iter) break;
        if (P.lead_iters >= 0 ? it >= P.lead_iters : code == RVE_OK) break;
    }
    // the hand-over evaluation's own residual, by every warp
    cl.sync();
    const Verdict v = residual_verdict(sh, pt, (int)(it & 3), it, thresh2, want_k, P.max_iter);
    r2 = {v.r2h, v.r2l};
    k2 = {v.k2h, v.k2l};
    status = v.code >= 0 ? v.code : RVE_PENDING;
    // the double-float displacement for the FP32 kernel and the output
    const int t = (int)(it & 1);
    const float4 *Hc = U0 + 2 * t * part_cap, *Lc = Hc + part_cap;
    for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
        const int i = pt.f0 + k;
        const float4 ph = Hc[k], pl = Lc[k];
        uh[i] = ph.x; uh[n + i] = ph.y; uh[2 * n + i] = ph.z;
        ul[i] = pl.x; ul[n + i] = pl.y; ul[2 * n + i] = pl.z;
        const float4 vhk = st.VH[k], vlk = st.VL[k], ay = st.AY[k];
        vh[i] = vhk.x; vh[n + i] = vhk.y; vh[2 * n + i] = vhk.z;
        vl[i] = vlk.x; vl[n + i] = vlk.y; vl[2 * n + i] = vlk.z;
        ah[i] = vhk.w; ah[n + i] = ay.x; ah[2 * n + i] = ay.y;
        al[i] = vlk.w; al[n + i] = ay.z; al[2 * n + i] = ay.w;
    }
}

// End of a mixed solve of RVE p: the final displacement (FP64 output; the
// double-float displacement plus the FP32 increment Qfin when given), the
// FP64 stress sum split across the cluster, and the per-RVE outputs.
__device__ void mixed_finish(cg::cluster_group &cl, MixedShared &sh, const DevMesh &M, const DevState &S,
                             const DevResults &O, const SolveParams &P, int p, const RveDesc &R,
                             const Part &pt, const double *F, const float4 *Qfin, int status, int64_t it,
                             df r2, df k2, double f_ref) {
    const int n = R.n_nodes, m = pt.m();
    const int64_t n0 = R.node0, b3 = 3 * n0;
    const float *uh = S.uh + b3, *ul = S.ul + b3;
    double *xg = S.xg + b3;
    const bool want_k = P.want_ke != 0;
    const int fin = Qfin ? 0 : -1;
    // ---- final displacement (FP64 output) and positions for the stress ----
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int i = pt.gidx(k);
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
        if (fin >= 0 && k < pt.nfr) d = Qfin[k];
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
        O.ke[p] = want_k ? df_to_double(k2) : 0.0;
    }
    cl.sync();
}

// ---------------------------------------------------------------------------
// lead kernel: setup (Algorithm 1 lines up to the loop) and the double-float
// iterations
// ---------------------------------------------------------------------------
template <bool STAGE>
__device__ void lead_rve(cg::cluster_group &cl, MixedShared &sh, const DevMesh &M, const DevState &S,
                         const DevResults &O, const SolveParams &P, int p, float4 *Pl, float4 *Q0,
                         const Staged &st, int part_cap, int elem_cap, int slot_cap, int &rb) {
    const RveDesc R = M.rve[p];
    const Part pt = make_part(M, R, p, (int)cl.block_rank(), (int)cl.num_blocks());
    const int n = R.n_nodes, m = pt.m();
    const int64_t n0 = R.node0, b3 = 3 * n0;
    const int32_t *rowptr = M.rowptr + R.rp0;
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = P.F[9 * (int64_t)p + k];
    float *uh = S.uh + b3, *ul = S.ul + b3, *vh = S.vh + b3, *vl = S.vl + b3;
    float *ah = S.ah + b3, *al = S.al + b3, *fg = S.fg + b3;
    const float *imh = M.imh + n0, *iml = M.iml + n0;
    const bool want_k = P.want_ke != 0;
    double f_ref = 0.0;
    int64_t it = 0;
    if (P.resume) {
        // resume launch: only RVEs the FP32 phase handed back, from the state
        // it left (double-float displacement, velocity, acceleration)
        const int st0 = O.status[p];
        f_ref = O.f_ref[p];
        it = O.iters[p];
        cl.sync();  // every CTA has read the status before rank 0 rewrites it
        if (st0 != RVE_STALLED) return;
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const int i = pt.gidx(k);
            Pl[k] = make_float4(uh[i], uh[n + i], uh[2 * n + i], 0.f);
            Q0[k] = make_float4(ul[i], ul[n + i], ul[2 * n + i], 0.f);
        }
        cl.sync();
    } else {
    // affine displacement (F - I) X for f_ref, and the initial displacement
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int i = pt.gidx(k);
        const double X[3] = {M.X0[n0 + i], M.X1[n0 + i], M.X2[n0 + i]};
        const double *uw[3] = {S.u0 + n0, S.u1 + n0, S.u2 + n0};
        df ua[3];
        const bool fixed = k >= pt.nfr;
        for (int r = 0; r < 3; ++r) {
            const double xa = dadd(dadd(dmul(F[3 * r], X[0]), dmul(F[3 * r + 1], X[1])), dmul(F[3 * r + 2], X[2]));
            const double uaff = dsub(xa, X[r]);
            ua[r] = df_from_double(uaff);
            double u;
            if (fixed || P.init == 1) u = uaff;
            else if (P.init == 2) u = uw[r][i];
            else u = 0.0;
            const df ud = df_from_double(u);
            uh[r * n + i] = ud.hi;
            ul[r * n + i] = ud.lo;
        }
        Pl[k] = make_float4(ua[0].hi, ua[1].hi, ua[2].hi, 0.f);
        Q0[k] = make_float4(ua[0].lo, ua[1].lo, ua[2].lo, 0.f);
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
    rb = (rb + 1) % kLeadBufs;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int i = pt.gidx(k);
        Pl[k] = make_float4(uh[i], uh[n + i], uh[2 * n + i], 0.f);
        Q0[k] = make_float4(ul[i], ul[n + i], ul[2 * n + i], 0.f);
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
    rb = (rb + 1) % kLeadBufs;
    f_ref = f_aff > f0 ? f_aff : f0;
    }
    const df thresh2 = df_from_double(dmul(dmul(P.tol, f_ref), dmul(P.tol, f_ref)));
    // a resumed RVE runs in double-float until it converges
    const df lead2 = P.resume ? thresh2 : df_from_double(dmul(dmul(P.lead_tol, f_ref), dmul(P.lead_tol, f_ref)));
    const int64_t lead_iters = P.resume ? -1 : P.lead_iters;
    const double dt64 = dmul(P.alpha, R.dtc);
    const df dt = df_from_double(dt64), hdt = df_from_double(dmul(0.5, dt64));
    const df cdf = df_from_double(R.c);

    const int64_t it0 = it;
    int status = RVE_PENDING;
    df r2 = df_from(0.f), k2 = df_from(0.f);
    if (STAGE) {
        SolveParams Q = P;
        Q.lead_iters = lead_iters;
        for (;;) {
            lead_loop_staged(cl, sh, M, S, R, pt, Q, Pl, st, part_cap, elem_cap, slot_cap, lead2, thresh2,
                             dt, hdt, cdf, it, status, r2, k2);
            // The loop stops two evaluations after the tested one; when
            // resuming, the state it stops at must itself be converged, else
            // the iteration goes on from that state.
            if (!P.resume || status != RVE_PENDING) break;
            for (int k = threadIdx.x; k < m; k += blockDim.x) {
                const int i = pt.gidx(k);
                Pl[k] = make_float4(uh[i], uh[n + i], uh[2 * n + i], 0.f);
                Q0[k] = make_float4(ul[i], ul[n + i], ul[2 * n + i], 0.f);
            }
            cl.sync();
        }
    } else {
    // L lanes share a node's edges; lane 0 of group k owns node k's state in
    // every phase, so consecutive phases need no barrier between them.
    int L = 1;
    while (L < 4 && (int)blockDim.x >= 2 * L * R.part_free_max) L *= 2;
    const int sub = threadIdx.x & (L - 1), grp = threadIdx.x / L, ngrp = blockDim.x / L;
    for (;;) {
        for (int k = grp; k < pt.nfr; k += ngrp) {
            if (sub != 0) continue;
            const int i = pt.f0 + k;
            df u[3];
            for (int c = 0; c < 3; ++c) {
                df v = {vh[c * n + i], vl[c * n + i]};
                const df a = {ah[c * n + i], al[c * n + i]};
                v = df_add(v, df_mul(hdt, a));
                u[c] = df_add({uh[c * n + i], ul[c * n + i]}, df_mul(dt, v));
                vh[c * n + i] = v.hi; vl[c * n + i] = v.lo;
                uh[c * n + i] = u[c].hi; ul[c * n + i] = u[c].lo;
            }
            Pl[k] = make_float4(u[0].hi, u[1].hi, u[2].hi, 0.f);
            Q0[k] = make_float4(u[0].lo, u[1].lo, u[2].lo, 0.f);
        }
        cl.sync();
        float rs = 0.f, kes = 0.f;
        for (int kb = 0; kb < pt.nfr; kb += ngrp) {
            const int k = kb + grp;
            const bool valid = k < pt.nfr;
            df g[3] = {df_from(0.f), df_from(0.f), df_from(0.f)};
            if (valid) gather_df(M, R, rowptr, sh, pt, k, Pl, Q0, 0, g[0], g[1], g[2], sub, L);
            df_group_sum(g[0], g[1], g[2], L);
            if (!valid || sub != 0) continue;
            const int i = pt.f0 + k;
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
        rb = (rb + 1) % kLeadBufs;
        ++it;
        if (!isfinite(r2.hi)) { status = RVE_NAN; break; }
        if (df_le(r2, thresh2)) { status = RVE_OK; break; }
        if (it >= P.max_iter) { status = RVE_MAXITER; break; }
        if (lead_iters >= 0 ? it >= lead_iters : df_le(r2, lead2)) break;
    }
    }
    if (P.resume) {
        if (pt.me == 0 && threadIdx.x == 0) O.lead[p] += it - it0;
        mixed_finish(cl, sh, M, S, O, P, p, R, pt, F, nullptr, status, it, r2, k2, f_ref);
        return;
    }
    if (pt.me == 0 && threadIdx.x == 0) {
        O.iters[p] = it;
        O.lead[p] = it;
        O.status[p] = status;
        O.f_ref[p] = f_ref;
        O.rel_res[p] = df_to_double(r2);  // squared residual, finished by the FP32 kernel
        O.ke[p] = want_k ? df_to_double(k2) : 0.0;
    }
    cl.sync();
}

// ---------------------------------------------------------------------------
// FP32 kernel: increment iterations, reference refreshes, final state, stress
// ---------------------------------------------------------------------------
// The next iteration's partial velocity update (Algorithm 1: v += dt/2 a)
// and displacement increment (u += dt v, as an increment on top of d) for one
// node, from its velocity w and acceleration a after this iteration.
__device__ __forceinline__ void next_increment(float w0, float w1, float w2, float a0, float a1, float a2,
                                               const float4 &d, float hdtf, float dtf, float4 &sv,
                                               float2 &sa, float4 &next) {
    const float v0 = w0 + hdtf * a0, v1 = w1 + hdtf * a1, v2 = w2 + hdtf * a2;
    sv = make_float4(v0, v1, v2, a0);
    sa = make_float2(a1, a2);
    next = make_float4(d.x + dtf * v0, d.y + dtf * v1, d.z + dtf * v2, 0.f);
}

template <bool STAGE>
__device__ void fp32_rve(cg::cluster_group &cl, MixedShared &sh, const DevMesh &M, const DevState &S,
                         const DevResults &O, const SolveParams &P, int p, float4 *Pl,
                         float4 *const *Qb, float4 *SVs, float2 *SAs, const Staged &st, int elem_cap,
                         int slot_cap, uint32_t bstride) {
    const RveDesc R = M.rve[p];
    const Part pt = make_part(M, R, p, (int)cl.block_rank(), (int)cl.num_blocks());
    const int n = R.n_nodes, m = pt.m();
    const int64_t n0 = R.node0, b3 = 3 * n0;
    const int32_t *rowptr = M.rowptr + R.rp0;
    // velocity (+ a.x) and a.yz of the own free nodes: shared memory with the
    // element table; otherwise global (L2-resident) arrays, which keeps the
    // unstaged kernel's shared memory at 96 bytes per node
    float4 *SV = STAGE ? SVs : S.sv + n0 + pt.f0;
    float2 *SA = STAGE ? SAs : S.sa + n0 + pt.f0;
    const float *Xh = M.Xh + b3, *Xl = M.Xl + b3;
    float *uh = S.uh + b3, *ul = S.ul + b3, *vh = S.vh + b3, *ah = S.ah + b3, *fg = S.fg + b3;
    const float *imh = M.imh + n0;
    const bool want_k = P.want_ke != 0;
    double F[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) F[k] = P.F[9 * (int64_t)p + k];

    int status = O.status[p];
    int64_t it = O.iters[p];
    const double f_ref = O.f_ref[p];
    df r2 = df_from_double(O.rel_res[p]);
    df k2 = df_from_double(O.ke[p]);
    int fin = -1;  // increment buffer holding the final state, -1: none
    cl.sync();     // every CTA has read the lead's results before rank 0 rewrites them

    if (status == RVE_PENDING) {
        const df thresh2 = df_from_double(dmul(dmul(P.tol, f_ref), dmul(P.tol, f_ref)));
        const double dt64 = dmul(P.alpha, R.dtc);
        const float dtf = (float)dt64, hdtf = (float)dmul(0.5, dt64), cf = (float)R.c;
        const int K = P.rebase_every > 0 ? P.rebase_every : 512;
        // lanes per node: with the element table one (element forces are spread
        // over all threads, node sums are short); otherwise as many as the CTA
        // size allows for this RVE's largest part. Node k's velocity and
        // acceleration are owned by lane 0 of group k in every phase, so
        // consecutive phases need no barrier between them.
        int lanes = 1;
        while (!STAGE && lanes < 4 && (int)blockDim.x >= 2 * lanes * R.part_free_max) lanes *= 2;
        const int L = lanes;
        const int sub = threadIdx.x & (L - 1), grp = threadIdx.x / L, ngrp = blockDim.x / L;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const bool test_warp = warp == (int)(blockDim.x >> 5) - 1;
        // x_ref = X + u (FP32 rounding of the double-float sum), increments zero;
        // g_ref = fg from the lead's last force evaluation at exactly this state
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const int i = pt.gidx(k);
            float xr[3];
            for (int c = 0; c < 3; ++c)
                xr[c] = df_add({Xh[c * n + i], Xl[c * n + i]}, {uh[c * n + i], ul[c * n + i]}).hi;
            Pl[k] = make_float4(xr[0], xr[1], xr[2], 0.f);
            for (int b = 0; b < kBufs; ++b) Qb[b][k] = make_float4(0.f, 0.f, 0.f, 0.f);
            // velocity and acceleration of own free nodes live in shared memory
            // (rewritten every iteration; global stores would miss L1 each time)
            if (k < pt.nfr) {
                SV[k] = make_float4(vh[i], vh[n + i], vh[2 * n + i], ah[i]);
                SA[k] = make_float2(ah[n + i], ah[2 * n + i]);
                if (STAGE) st.SG[k] = make_float4(fg[i], fg[n + i], fg[2 * n + i], imh[i]);
            }
        }
        if (STAGE) {
            element_counts(M, R, pt, rowptr, st);
            __syncthreads();
            if (threadIdx.x == 0) element_offsets(sh, pt, st);
        }
        if (threadIdx.x == 0) {
            sh.st_h = INFINITY;
            sh.st_l = 0.f;
            sh.st_e = it;
        }
        cl.sync();
        int n_el = 0;
        if (STAGE) {
            // The capacities are sized on the host for every part. Should a
            // part not fit, every CTA of the cluster sees it (so all leave the
            // loop together) and the RVE is reported failed.
            bool over = false;
            for (int r = 0; r < pt.C; ++r)
                over |= *cl.map_shared_rank(&sh.elems, r) > elem_cap ||
                        *cl.map_shared_rank(&sh.slots, r) > slot_cap;
            if (over) status = RVE_NAN;
            else element_setup(sh, M, R, pt, rowptr, Pl, Qb[0], st, true);
            n_el = sh.elems;
        }
        const int64_t first = it;  // evaluation index of the first FP32 iteration
        int64_t chk = first;       // next evaluation whose residual is still untested
        int chkb = 0;              // its buffer
        // the verdict the testing warp wrote in the previous iteration
        bool vpend = false;
        int64_t veval = 0;
        int vbuf = 0;
        int since = 0;
        const int32_t *colp = M.col_part + R.csr0;
        const float2 *eafp = M.eaf + R.csr0;
        // Partial velocity update and displacement increment of the first
        // iteration; every later one is done by the node's owner right after
        // the node's velocity update of the previous iteration (the values are
        // still in registers), so an iteration begins at the barrier.
        for (int k = grp; k < pt.nfr; k += ngrp) {
            if (sub != 0) continue;
            const float4 va = SV[k];
            const float2 a12 = SA[k];
            next_increment(va.x, va.y, va.z, va.w, a12.x, a12.y, make_float4(0.f, 0.f, 0.f, 0.f),
                           hdtf, dtf, SV[k], SA[k], Qb[0][k]);
        }
        int b = 0;  // buffer of evaluation nidx
        float part_rs = 0.f, part_ke = 0.f;  // this thread's partials of evaluation nidx-1
        int part_b = -1;                     // and their buffer (-1: none yet)
        for (int64_t nidx = first; status == RVE_PENDING; ++nidx, b = (b + 1 == kBufs ? 0 : b + 1)) {
            const int bn = b + 1 == kBufs ? 0 : b + 1;  // buffer of evaluation nidx + 1
            const int bp = b == 0 ? kBufs - 1 : b - 1;  // buffer of evaluation nidx - 1
            const bool rebase = since >= K;
            cluster_arrive();
            // While the barrier completes: the per-warp residual partials of
            // evaluation nidx-1 go to this CTA's buffer, and evaluation nidx-3
            // (whose partials every CTA has published one barrier ago) is
            // tested by one warp per CTA, whose verdict the others read after
            // the next barrier; before a rebase by every warp. Buffers rotate
            // through five, so the state of a tested evaluation is intact
            // until its verdict is read.
            if (part_b >= 0) {
                for (int o = 16; o > 0; o >>= 1) part_rs += __shfl_xor_sync(0xffffffffu, part_rs, o);
                if (want_k)
                    for (int o = 16; o > 0; o >>= 1) part_ke += __shfl_xor_sync(0xffffffffu, part_ke, o);
                if (lane == 0) {
                    sh.own[part_b][0][warp] = part_rs;
                    if (want_k) sh.own[part_b][1][warp] = part_ke;
                }
            }
            bool tnow = false;
            int64_t teval = 0;
            int tbuf = 0;
            Verdict mine = {-1, 0.f, 0.f, 0.f, 0.f};
            if (chk <= nidx - 3) {
                if (rebase || test_warp) mine = residual_verdict(sh, pt, chkb, chk + 1, thresh2, want_k, P.max_iter);
                if (!rebase && test_warp && lane == 0) {
                    // Stall check: the squared residual must reach a quarter of
                    // its reference value within stall_window evaluations,
                    // else the RVE goes back to the double-float kernel (the
                    // FP32 increments have hit their rounding floor). Every
                    // CTA's testing warp sees the same verdicts, so all agree.
                    if (mine.code < 0 && P.stall_window > 0) {
                        const df r2c = {mine.r2h, mine.r2l};
                        if (df_le(r2c, {0.25f * sh.st_h, 0.25f * sh.st_l})) {
                            sh.st_h = r2c.hi;
                            sh.st_l = r2c.lo;
                            sh.st_e = chk;
                        } else if (chk - sh.st_e >= P.stall_window) {
                            mine.code = RVE_STALLED;
                        }
                    }
                    sh.vd[b] = mine;
                }
                tnow = true; teval = chk; tbuf = chkb;
                ++chk;
                chkb = chkb + 1 == kBufs ? 0 : chkb + 1;
            }
            cluster_wait();
            Verdict stopv = {-1, 0.f, 0.f, 0.f, 0.f};
            int64_t seval = 0;
            int sbuf = 0;
            if (vpend) {
                const Verdict v = sh.vd[bp];
                if (v.code >= 0) { stopv = v; seval = veval; sbuf = vbuf; }
            }
            vpend = false;
            if (stopv.code < 0 && rebase) {
                // the reference moves: every earlier evaluation is tested first
                if (tnow && mine.code >= 0) { stopv = mine; seval = teval; sbuf = tbuf; }
                if (stopv.code < 0 && chk == nidx - 2) {  // published one barrier ago
                    mine = residual_verdict(sh, pt, chkb, chk + 1, thresh2, want_k, P.max_iter);
                    if (mine.code >= 0) { stopv = mine; seval = chk; sbuf = chkb; }
                    ++chk;
                    chkb = chkb + 1 == kBufs ? 0 : chkb + 1;
                }
                if (stopv.code < 0 && chk == nidx - 1) {  // published in this barrier's window
                    cl.sync();
                    mine = residual_verdict(sh, pt, chkb, chk + 1, thresh2, want_k, P.max_iter);
                    if (mine.code >= 0) { stopv = mine; seval = chk; sbuf = chkb; }
                    ++chk;
                    chkb = chkb + 1 == kBufs ? 0 : chkb + 1;
                }
            }
            if (stopv.code == RVE_STALLED) {
                // Hand back at the end of evaluation nidx-1, whose state is
                // complete: displacement = double-float base + its increment
                // (buffer bp), acceleration a, full-step velocity = SV - dt/2 a.
                const float4 *inc = Qb[bp];
                for (int k = grp; k < pt.nfr; k += ngrp) {
                    if (sub != 0) continue;
                    const int i = pt.f0 + k;
                    const float4 d = inc[k], va = SV[k];
                    const float2 ay = SA[k];
                    const float dd[3] = {d.x, d.y, d.z}, vv[3] = {va.x, va.y, va.z}, aa[3] = {va.w, ay.x, ay.y};
                    for (int c = 0; c < 3; ++c) {
                        const df u = df_add_f({uh[c * n + i], ul[c * n + i]}, dd[c]);
                        uh[c * n + i] = u.hi;
                        ul[c * n + i] = u.lo;
                        S.vh[b3 + c * n + i] = vv[c] - hdtf * aa[c];
                        S.vl[b3 + c * n + i] = 0.f;
                        S.ah[b3 + c * n + i] = aa[c];
                        S.al[b3 + c * n + i] = 0.f;
                    }
                }
                status = RVE_STALLED;
                it = nidx - 1;
                break;
            }
            if (stopv.code >= 0) {
                status = stopv.code;
                fin = sbuf;
                it = seval + 1;
                r2 = {stopv.r2h, stopv.r2l};
                k2 = {stopv.k2h, stopv.k2l};
                break;
            }
            float4 *cur = Qb[b];
            float rs = 0.f, kes = 0.f;
            if (rebase) {
                // fold the increment into the double-float displacement; stage
                // double-float displacements (hi in Pl, lo in buffer b)
                for (int k = threadIdx.x; k < m; k += blockDim.x) {
                    const int i = pt.gidx(k);
                    const float4 d = cur[k];
                    const float dd[3] = {d.x, d.y, d.z};
                    df u[3];
                    for (int c = 0; c < 3; ++c) {
                        u[c] = {uh[c * n + i], ul[c * n + i]};
                        if (k < pt.nfr) {
                            u[c] = df_add_f(u[c], dd[c]);
                            uh[c * n + i] = u[c].hi; ul[c * n + i] = u[c].lo;
                        }
                    }
                    Pl[k] = make_float4(u[0].hi, u[1].hi, u[2].hi, 0.f);
                    cur[k] = make_float4(u[0].lo, u[1].lo, u[2].lo, 0.f);
                }
                cl.sync();
                for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
                    const int i = pt.f0 + k;
                    df g[3];
                    gather_df(M, R, rowptr, sh, pt, k, Pl, cur, b, g[0], g[1], g[2]);
                    fg[i] = g[0].hi; fg[n + i] = g[1].hi; fg[2 * n + i] = g[2].hi;
                    if (STAGE) st.SG[k] = make_float4(g[0].hi, g[1].hi, g[2].hi, imh[i]);
                }
                cl.sync();
                // back to FP32 reference positions and zero increments
                for (int k = threadIdx.x; k < m; k += blockDim.x) {
                    const int i = pt.gidx(k);
                    float xr[3];
                    for (int c = 0; c < 3; ++c)
                        xr[c] = df_add({Xh[c * n + i], Xl[c * n + i]}, {uh[c * n + i], ul[c * n + i]}).hi;
                    Pl[k] = make_float4(xr[0], xr[1], xr[2], 0.f);
                    cur[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
                cl.sync();
                if (STAGE) element_setup(sh, M, R, pt, rowptr, Pl, Qb[0], st, false);
                for (int k = grp; k < pt.nfr; k += ngrp) {
                    if (sub != 0) continue;
                    const int i = pt.f0 + k;
                    const float im = imh[i];
                    const float4 va = SV[k];
                    const float g0 = fg[i], g1 = fg[n + i], g2 = fg[2 * n + i];
                    const float a0 = g0 * im - cf * va.x, a1 = g1 * im - cf * va.y,
                                a2 = g2 * im - cf * va.z;
                    const float w0 = va.x + hdtf * a0, w1 = va.y + hdtf * a1, w2 = va.z + hdtf * a2;
                    next_increment(w0, w1, w2, a0, a1, a2, cur[k], hdtf, dtf, SV[k], SA[k], Qb[bn][k]);
                    rs += g0 * g0 + g1 * g1 + g2 * g2;
                    if (want_k) kes += 0.5f * (w0 * w0 + w1 * w1 + w2 * w2) / im;
                }
                since = 0;
            } else {
                vpend = tnow; veval = teval; vbuf = tbuf;
                const uint32_t boff = (uint32_t)b * bstride;
                if (STAGE) {
                    // element forces, spread evenly over the CTA's threads
                    for (int u = threadIdx.x; u < n_el; u += blockDim.x) {
                        const float4 k0 = st.K0[u], k1 = st.K1[u];
                        const float4 qa = ld_local(st.EI[u] + boff);
                        const uint32_t ab = __float_as_uint(k1.w);
                        const float4 qb = (ab & 1u) ? ld_cluster((ab & ~1u) + boff) : ld_local(ab + boff);
                        float t0 = 0.f, t1 = 0.f, t2 = 0.f;
                        edge_increment_slot(qa, qb, k0, k1, t0, t1, t2);
                        st.TF[u] = make_float4(t0, t1, t2, 0.f);
                    }
                    __syncthreads();
                    // node sums in CSR row order, then the velocity update
                    for (int k = threadIdx.x; k < pt.nfr; k += blockDim.x) {
                        const int deg = st.SD[k];
                        int sl = st.SS[k >> 5] + (k & 31);
                        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
                        for (int j = 0; j < deg; ++j, sl += 32) {
                            const uint32_t w = st.NS[sl];
                            const float4 t = st.TF[w >> 1];
                            if (w & 1u) { g0 -= t.x; g1 -= t.y; g2 -= t.z; }
                            else { g0 += t.x; g1 += t.y; g2 += t.z; }
                        }
                        const float4 gr = st.SG[k];
                        g0 += gr.x; g1 += gr.y; g2 += gr.z;
                        const float im = gr.w;
                        const float4 va = SV[k];
                        float w0 = va.x, w1 = va.y, w2 = va.z;
                        const float a0 = g0 * im - cf * w0;
                        const float a1 = g1 * im - cf * w1;
                        const float a2 = g2 * im - cf * w2;
                        w0 += hdtf * a0; w1 += hdtf * a1; w2 += hdtf * a2;
                        next_increment(w0, w1, w2, a0, a1, a2, cur[k], hdtf, dtf, SV[k], SA[k], Qb[bn][k]);
                        rs += g0 * g0 + g1 * g1 + g2 * g2;
                        if (want_k) kes += 0.5f * (w0 * w0 + w1 * w1 + w2 * w2) / im;
                    }
                } else {
                    // L lanes share a node's edges (lane s takes edges s, s+L, ...,
                    // two at a time) and combine with shuffles; L is fixed per RVE
                    // so its result does not depend on the launch it runs in.
                    for (int kb = 0; kb < pt.nfr; kb += ngrp) {
                        const int k = kb + grp;
                        const bool valid = k < pt.nfr;
                        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
                        if (valid) {
                            const float4 qi = cur[k];
                            const int i = pt.f0 + k;
                            const float4 pi = Pl[k];
                            const int end = rowptr[i + 1];
                            int e = rowptr[i] + sub;
                            for (; e + L < end; e += 2 * L) {
                                const int ca = __ldg(colp + e), cb = __ldg(colp + e + L);
                                const float2 ea = __ldg(eafp + e), eb = __ldg(eafp + e + L);
                                const int ra = ca >> 16, la = ca & 0xffff, rb2 = cb >> 16, lb = cb & 0xffff;
                                const float4 pa = ra == pt.me ? Pl[la] : sh.P[ra][la];
                                const float4 qa = ra == pt.me ? cur[la] : sh.Q[b][ra][la];
                                const float4 pb = rb2 == pt.me ? Pl[lb] : sh.P[rb2][lb];
                                const float4 qb = rb2 == pt.me ? cur[lb] : sh.Q[b][rb2][lb];
                                edge_increment(pi, qi, pa, qa, ea, g0, g1, g2);
                                edge_increment(pi, qi, pb, qb, eb, g0, g1, g2);
                            }
                            if (e < end) {
                                const int ca = __ldg(colp + e);
                                const float2 ea = __ldg(eafp + e);
                                const int ra = ca >> 16, la = ca & 0xffff;
                                const float4 pa = ra == pt.me ? Pl[la] : sh.P[ra][la];
                                const float4 qa = ra == pt.me ? cur[la] : sh.Q[b][ra][la];
                                edge_increment(pi, qi, pa, qa, ea, g0, g1, g2);
                            }
                        }
                        for (int o = 1; o < L; o <<= 1) {
                            g0 += __shfl_xor_sync(0xffffffffu, g0, o);
                            g1 += __shfl_xor_sync(0xffffffffu, g1, o);
                            g2 += __shfl_xor_sync(0xffffffffu, g2, o);
                        }
                        if (valid && sub == 0) {
                            const int i = pt.f0 + k;
                            g0 += fg[i]; g1 += fg[n + i]; g2 += fg[2 * n + i];
                            const float im = imh[i];
                            const float4 va = SV[k];
                            float w0 = va.x, w1 = va.y, w2 = va.z;
                            const float a0 = g0 * im - cf * w0;
                            const float a1 = g1 * im - cf * w1;
                            const float a2 = g2 * im - cf * w2;
                            w0 += hdtf * a0; w1 += hdtf * a1; w2 += hdtf * a2;
                            next_increment(w0, w1, w2, a0, a1, a2, cur[k], hdtf, dtf, SV[k], SA[k],
                                           Qb[bn][k]);
                            rs += g0 * g0 + g1 * g1 + g2 * g2;
                            if (want_k) kes += 0.5f * (w0 * w0 + w1 * w1 + w2 * w2) / im;
                        }
                    }
                }
            }
            // this evaluation's partials are published in the next barrier's window
            part_rs = rs;
            part_ke = kes;
            part_b = b;
            ++since;
        }
    }

    if (status == RVE_STALLED) {
        // handed back to the double-float kernel (resume launch), which
        // finishes the solve and writes every output
        if (pt.me == 0 && threadIdx.x == 0) {
            O.iters[p] = it;
            O.status[p] = RVE_STALLED;
        }
        cl.sync();
        return;
    }
    mixed_finish(cl, sh, M, S, O, P, p, R, pt, F, fin >= 0 ? Qb[fin] : nullptr, status, it, r2, k2, f_ref);
}

}  // namespace

template <bool STAGE>
__global__ void __launch_bounds__(512, 1) dr_mixed_lead_kernel(DevMesh M, DevState S, DevResults O,
                                                            SolveParams P, int part_cap, int free_cap,
                                                            int elem_cap, int slot_cap) {
    extern __shared__ __align__(16) float4 dsm[];
    __shared__ MixedShared sh;
    cg::cluster_group cl = cg::this_cluster();
    float4 *Pl = dsm, *Q0 = dsm + part_cap;
    float4 *Qb[kBufs];
    for (int b = 0; b < kBufs; ++b) Qb[b] = Q0;
    Staged st = {};
    if (STAGE) {
        // layout as in mixed_lead_smem: two displacement buffers, velocity and
        // acceleration, then the tables
        st.VH = dsm + 4 * (size_t)part_cap;
        st.VL = st.VH + free_cap;
        st.AY = st.VL + free_cap;
        char *base = reinterpret_cast<char *>(st.AY + free_cap);
        st.K0 = reinterpret_cast<float4 *>(base);
        base += 16 * (size_t)elem_cap;
        st.K1 = reinterpret_cast<float4 *>(base);
        base += 16 * (size_t)elem_cap;
        st.KA = reinterpret_cast<float4 *>(base);
        base += 16 * (size_t)elem_cap;
        st.TA = reinterpret_cast<float4 *>(base);
        base += 16 * (size_t)elem_cap;
        st.TB = reinterpret_cast<float2 *>(base);
        base += 8 * (size_t)elem_cap;
        st.NS = reinterpret_cast<uint32_t *>(base);
        base += 4 * (size_t)slot_cap;
        st.SD = reinterpret_cast<int *>(base);
        base += 4 * (size_t)free_cap;
        st.EB = reinterpret_cast<int *>(base);
        base += 4 * (size_t)free_cap;
        st.SS = reinterpret_cast<int *>(base);
    }
    map_remote(cl, sh, Pl, Qb, (int)cl.num_blocks());
    int rb = 0;
    for (;;) {
        const int item = next_item(cl, sh, P.counter + (P.resume ? 2 : 0));
        if (item >= P.queue_len) return;
        lead_rve<STAGE>(cl, sh, M, S, O, P, P.queue[item], Pl, Q0, st, part_cap, elem_cap, slot_cap, rb);
    }
}

template <bool STAGE>
__global__ void __launch_bounds__(512, 1) dr_mixed_fp32_kernel(DevMesh M, DevState S, DevResults O,
                                                               SolveParams P, int part_cap,
                                                               int free_cap, int elem_cap,
                                                               int slot_cap) {
    extern __shared__ __align__(16) float4 dsm[];
    __shared__ MixedShared sh;
    cg::cluster_group cl = cg::this_cluster();
    float4 *Pl = dsm;
    float4 *Qb[kBufs];
    for (int b = 0; b < kBufs; ++b) Qb[b] = dsm + (1 + b) * part_cap;
    float4 *SV = dsm + (1 + kBufs) * part_cap;
    float2 *SA = reinterpret_cast<float2 *>(dsm + (2 + kBufs) * part_cap);
    Staged st = {};
    if (STAGE) {
        // layout as in mixed_fp32_smem
        char *base = reinterpret_cast<char *>(dsm) + align16(kFp32NodeBytes * part_cap);
        st.SG = reinterpret_cast<float4 *>(base);
        base += 16 * (size_t)free_cap;
        st.K0 = reinterpret_cast<float4 *>(base);
        base += 16 * (size_t)elem_cap;
        st.K1 = reinterpret_cast<float4 *>(base);
        base += 16 * (size_t)elem_cap;
        st.TF = reinterpret_cast<float4 *>(base);
        base += 16 * (size_t)elem_cap;
        st.EI = reinterpret_cast<uint32_t *>(base);
        base += 4 * (size_t)elem_cap;
        st.NS = reinterpret_cast<uint32_t *>(base);
        base += 4 * (size_t)slot_cap;
        st.SD = reinterpret_cast<int *>(base);
        base += 4 * (size_t)free_cap;
        st.EB = reinterpret_cast<int *>(base);
        base += 4 * (size_t)free_cap;
        st.SS = reinterpret_cast<int *>(base);
    }
    map_remote(cl, sh, Pl, Qb, (int)cl.num_blocks());
    const uint32_t bstride = (uint32_t)(sizeof(float4) * part_cap);
    for (;;) {
        const int item = next_item(cl, sh, P.counter + 1);
        if (item >= P.queue_len) return;
        fp32_rve<STAGE>(cl, sh, M, S, O, P, P.queue[item], Pl, Qb, SV, SA, st, elem_cap, slot_cap,
                        bstride);
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

// Raise a kernel's dynamic shared-memory limit (and allow 16-CTA clusters)
// once per device and size, so that launches recorded into a CUDA graph make
// no attribute calls of their own.
std::mutex g_prep_mutex;
std::map<std::pair<const void *, int>, int> g_prep_bytes;  // (kernel, device) -> limit set

template <class K>
void prepare(K kernel, size_t smem) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(g_prep_mutex);
    int &have = g_prep_bytes[{reinterpret_cast<const void *>(kernel), dev}];
    if (have < (int)smem || have == 0) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        have = std::max(have, (int)smem);
    }
}
}  // namespace

size_t mixed_fp32_smem(int part_cap, int free_cap, int elem_cap, int slot_cap, size_t limit) {
    const size_t plain = kFp32PlainNodeBytes * (size_t)part_cap;
    const size_t F = (size_t)free_cap, U = (size_t)elem_cap, S = (size_t)slot_cap;
    const size_t staged = align16(align16(kFp32NodeBytes * (size_t)part_cap) + 16 * F + 3 * 16 * U +
                                  4 * U + 4 * S + 2 * 4 * F + 4 * (F / 32 + 2));
    return staged <= limit ? staged : plain;
}

size_t mixed_lead_smem(int part_cap, int free_cap, int elem_cap, int slot_cap, size_t limit) {
    const size_t plain = kLeadPlainNodeBytes * (size_t)part_cap;
    const size_t F = (size_t)free_cap, U = (size_t)elem_cap, S = (size_t)slot_cap;
    const size_t staged =
        align16(2 * plain + 3 * 16 * F + 4 * 16 * U + 8 * U + 4 * S + 2 * 4 * F + 4 * (F / 32 + 2));
    return staged <= limit ? staged : plain;
}

bool mixed_staged(int lead, size_t smem, int part_cap) {
    return smem > (lead ? kLeadPlainNodeBytes : kFp32PlainNodeBytes) * (size_t)part_cap;
}

size_t mixed_plain_node_bytes(int lead) { return lead ? kLeadPlainNodeBytes : kFp32PlainNodeBytes; }

int launch_dr_mixed(const DevMesh &m, const DevState &s, const DevResults &r, const SolveParams &p,
                    int lead, int clusters, int parts, int block, size_t smem, int part_cap,
                    int free_cap, int elem_cap, int slot_cap, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = mixed_config(clusters, parts, block, smem, attr, st);
    const bool staged = mixed_staged(lead, smem, part_cap);
    cudaError_t e;
    if (lead && staged) {
        prepare(dr_mixed_lead_kernel<true>, smem);
        e = cudaLaunchKernelEx(&cfg, dr_mixed_lead_kernel<true>, m, s, r, p, part_cap, free_cap,
                               elem_cap, slot_cap);
    } else if (lead) {
        prepare(dr_mixed_lead_kernel<false>, smem);
        e = cudaLaunchKernelEx(&cfg, dr_mixed_lead_kernel<false>, m, s, r, p, part_cap, free_cap,
                               elem_cap, slot_cap);
    } else if (staged) {
        prepare(dr_mixed_fp32_kernel<true>, smem);
        e = cudaLaunchKernelEx(&cfg, dr_mixed_fp32_kernel<true>, m, s, r, p, part_cap, free_cap,
                               elem_cap, slot_cap);
    } else {
        prepare(dr_mixed_fp32_kernel<false>, smem);
        e = cudaLaunchKernelEx(&cfg, dr_mixed_fp32_kernel<false>, m, s, r, p, part_cap, free_cap,
                               elem_cap, slot_cap);
    }
    if (e != cudaSuccess) return (int)e;
    return (int)cudaGetLastError();
}

int occupancy_dr_mixed(int lead, int parts, int block, size_t smem, int part_cap) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = mixed_config(parts * 64, parts, block, smem, attr, nullptr);
    const bool staged = mixed_staged(lead, smem, part_cap);
    int n = 0;
    cudaError_t e;
    if (lead && staged) {
        prepare(dr_mixed_lead_kernel<true>, smem);
        e = cudaOccupancyMaxActiveClusters(&n, dr_mixed_lead_kernel<true>, &cfg);
    } else if (lead) {
        prepare(dr_mixed_lead_kernel<false>, smem);
        e = cudaOccupancyMaxActiveClusters(&n, dr_mixed_lead_kernel<false>, &cfg);
    } else if (staged) {
        prepare(dr_mixed_fp32_kernel<true>, smem);
        e = cudaOccupancyMaxActiveClusters(&n, dr_mixed_fp32_kernel<true>, &cfg);
    } else {
        prepare(dr_mixed_fp32_kernel<false>, smem);
        e = cudaOccupancyMaxActiveClusters(&n, dr_mixed_fp32_kernel<false>, &cfg);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace fe2
