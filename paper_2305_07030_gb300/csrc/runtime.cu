// Host runtime behind the C ABI of include/fe2.h: input validation, packing
// into the device layout of fe2_internal.h (free/fixed reordering, spatial
// parts per cluster CTA, node-centric CSR), size classes, the cost-ordered
// work queue, persistent launches and result readback.
//
// Algorithm 1 steps 1-3 (load mesh, build connectivity, transfer to the GPU)
// happen here once per batch; the mass matrix and time step are computed by
// create-time kernels, and every solver step runs in the solve kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <numeric>
#include <tuple>
#include <string>
#include <thread>
#include <vector>

#include "../../include/fe2.h"
#include "fe2_internal.h"

using namespace fe2;

namespace {

thread_local std::string g_err;

fe2_status fail(fe2_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

#define CUDA_TRY(expr)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (expr);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? FE2_ENOMEM : FE2_ECUDA,          \
                        std::string(#expr) + ": " + cudaGetErrorString(e_));               \
    } while (0)

template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count) {
        n = count;
        if (count == 0) return cudaSuccess;
        return cudaMalloc(&p, sizeof(T) * count);
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

// One size class: RVEs solved by one persistent launch.
struct SizeClass {
    int parts = 1;              // mixed: cluster size
    bool lead_staged = false;   // mixed: lead kernel with its element table
    bool fp32_staged = false;   // mixed: FP32 kernel with its element table
    int block_lead = 0;         // mixed: tuned CTA sizes (0 = default)
    int block_fp32 = 0;
    int smem_positions = 1;     // FP64: positions in shared memory
    bool fp64_cluster = false;  // FP64: one cluster of `parts` CTAs per RVE
    bool fp64_tsm = false;      // FP64 cluster: element table in shared memory
    bool fp64_ssm = false;      // FP64 cluster: free-node state in shared memory
    int fslot_max = 0;          // FP64 cluster: most element slots of one part
    size_t smem_bytes = 0;      // dynamic shared memory per CTA
    int part_max = 0;           // mixed: largest part (nodes)
    int free_max = 0;           // mixed: most free nodes in one part
    int elem_max = 0;           // mixed: most FP32-kernel table elements of one part
    int slot_max = 0;           // mixed: most FP32-kernel row slots of one part
    std::vector<int32_t> rves;  // in scheduling order
    int32_t queue_off = 0;      // offset of its queue in the device queue buffer
};

// One in-flight micro-batch of the serving interface: its own stream, queue
// and result staging, so submissions overlap on the device.
struct ServeSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int32_t *d_ids = nullptr;   // 2 * n_rve: submitted ids, then per-class queues
    int32_t *d_cnt = nullptr;   // work-queue heads, 2 per class
    double *d_F = nullptr;      // 9 * n_rve staged deformation gradients
    double *d_out = nullptr;    // 10 * n_rve: sigma (9) and rel_res per submitted id
    int64_t *d_it = nullptr;    // n_rve
    int32_t *d_st = nullptr;    // n_rve
    int32_t *h_ids = nullptr;   // pinned mirrors
    double *h_F = nullptr;
    double *h_out = nullptr;
    int64_t *h_it = nullptr;
    int32_t *h_st = nullptr;
    int n = 0;
    bool busy = false;
    double bytes = 0.0;         // working-set bytes it holds (admission)
};

constexpr int kServeSlots = 8;  // concurrent micro-batches of the serving interface

int env_int(const char *name, int dflt) {
    const char *v = std::getenv(name);
    return v && *v ? std::atoi(v) : dflt;
}

}  // namespace

struct fe2_batch {
    int32_t n_rve = 0;
    int64_t n_nodes = 0, n_elems = 0, n_csr = 0;
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    std::vector<RveDesc> rve;             // host copy
    std::vector<int64_t> perm_to_orig;    // permuted global -> caller global node
    std::vector<int32_t> part_free_max;   // per RVE, most free nodes in one part

    // device arrays
    DevBuf<RveDesc> d_rve;
    DevBuf<double> d_X, d_mass, d_EA_csr, d_L_csr, d_el_EA, d_el_L;
    DevBuf<float> d_Xh, d_Xl, d_imh, d_iml;
    DevBuf<int32_t> d_rowptr, d_col, d_col_part, d_part_off, d_el_a, d_el_b, d_csr_el;
    DevBuf<int32_t> d_fp_csr_slot, d_fp_part_slot;
    DevBuf<int4> d_fp_slot;
    DevBuf<double> d_ualt, d_fpt;
    DevBuf<float2> d_eaf, d_eaf_lo, d_sa;
    DevBuf<float4> d_sv;
    DevBuf<float4> d_dh, d_dl;
    DevBuf<double> d_u, d_v, d_a, d_xg, d_tf;
    DevBuf<float> d_uh, d_ul, d_vh, d_vl, d_ah, d_al, d_fg;
    DevBuf<double> d_F, d_sigma, d_rel, d_fref, d_ke, d_wint, d_wext, d_gp, d_fdp;
    DevBuf<int64_t> d_iters, d_lead;
    DevBuf<int32_t> d_status, d_queue, d_counters;
    DevBuf<double> d_naive;               // naive comparator scratch (first use)

    std::vector<SizeClass> classes_fp64, classes_mixed;
    bool solved = false;
    int32_t last_launches = 0;
    int32_t last_timed = 0;               // persistent launches bracketed by tev
    int last_energy = 0;                  // kinetic_energy option of the last batched solve
    cudaStream_t last_stream = nullptr;
    std::vector<cudaStream_t> side;       // forked streams for concurrent classes
    std::vector<cudaEvent_t> ev;
    std::vector<cudaEvent_t> tev;         // timing events around each class launch
    double *h_F = nullptr;                // pinned staging for F
    cudaEvent_t ev_F = nullptr;           // completion of the last F upload
    // cost-ordered queues from the previous solve's iteration counts
    cudaStream_t aux = nullptr;           // private stream for small copies
    cudaEvent_t ev_done = nullptr;        // end of the last batched solve
    int64_t *h_iters = nullptr;           // pinned
    int32_t *h_queue = nullptr;           // pinned, 2 * n_rve
    bool iters_known = false;
    // serving: micro-batch slots and the RVEs they hold
    std::vector<ServeSlot> slots;
    std::vector<uint8_t> in_flight;
    std::vector<int32_t> class_of_fp64, class_of_mixed;  // RVE -> class index
    // resident CTAs (FP64) or clusters (mixed) per launch shape, queried once
    // so that nothing but launches happens while a solve is captured
    std::map<std::tuple<int, int, int, size_t, int>, int> occ;
    // the batched solve as a CUDA graph, valid for the options it was
    // captured with (the kernels read F, queues and state from device memory)
    cudaGraphExec_t graph = nullptr;
    cudaStream_t cap = nullptr;           // private capture stream
    fe2_opts graph_opts = {};
    int graph_launches = 0, graph_timed = 0;

    DevMesh mesh() const {
        DevMesh m;
        m.rve = d_rve.p;
        m.X0 = d_X.p;
        m.X1 = d_X.p + n_nodes;
        m.X2 = d_X.p + 2 * n_nodes;
        m.Xh = d_Xh.p;
        m.Xl = d_Xl.p;
        m.mass = d_mass.p;
        m.imh = d_imh.p;
        m.iml = d_iml.p;
        m.rowptr = d_rowptr.p;
        m.col = d_col.p;
        m.col_part = d_col_part.p;
        m.part_off = d_part_off.p;
        m.EA = d_EA_csr.p;
        m.L = d_L_csr.p;
        m.eaf = d_eaf.p;
        m.eaf_lo = d_eaf_lo.p;
        m.dh = d_dh.p;
        m.dl = d_dl.p;
        m.el_a = d_el_a.p;
        m.el_b = d_el_b.p;
        m.el_EA = d_el_EA.p;
        m.el_L = d_el_L.p;
        m.csr_el = d_csr_el.p;
        m.fp_slot = d_fp_slot.p;
        m.fp_csr_slot = d_fp_csr_slot.p;
        m.fp_part_slot = d_fp_part_slot.p;
        return m;
    }
    DevState state() const {
        DevState s;
        s.u0 = d_u.p; s.u1 = d_u.p + n_nodes; s.u2 = d_u.p + 2 * n_nodes;
        s.v0 = d_v.p; s.v1 = d_v.p + n_nodes; s.v2 = d_v.p + 2 * n_nodes;
        s.a0 = d_a.p; s.a1 = d_a.p + n_nodes; s.a2 = d_a.p + 2 * n_nodes;
        s.uh = d_uh.p; s.ul = d_ul.p; s.vh = d_vh.p; s.vl = d_vl.p;
        s.ah = d_ah.p; s.al = d_al.p; s.fg = d_fg.p;
        s.xg = d_xg.p;
        s.tf = d_tf.p;
        s.sv = d_sv.p;
        s.gp = d_gp.p;
        s.ualt = d_ualt.p;
        s.fpt = d_fpt.p;
        s.fdp = d_fdp.p;
        s.sa = d_sa.p;
        return s;
    }
    DevResults results() const {
        DevResults r;
        r.sigma = d_sigma.p; r.iters = d_iters.p; r.rel_res = d_rel.p;
        r.status = d_status.p; r.f_ref = d_fref.p; r.ke = d_ke.p; r.lead = d_lead.p;
        r.wint = d_wint.p; r.wext = d_wext.p;
        return r;
    }
    void release() {
        d_rve.release(); d_X.release(); d_mass.release(); d_EA_csr.release(); d_L_csr.release();
        d_el_EA.release(); d_el_L.release(); d_Xh.release(); d_Xl.release(); d_imh.release();
        d_iml.release(); d_rowptr.release(); d_col.release(); d_col_part.release();
        d_part_off.release(); d_el_a.release(); d_el_b.release(); d_csr_el.release(); d_fp_csr_slot.release(); d_fp_part_slot.release(); d_fp_slot.release(); d_ualt.release(); d_fpt.release(); d_tf.release(); d_sv.release(); d_sa.release(); d_eaf.release();
        d_eaf_lo.release(); d_dh.release(); d_dl.release(); d_u.release(); d_v.release(); d_a.release(); d_xg.release();
        d_uh.release(); d_ul.release(); d_vh.release(); d_vl.release(); d_ah.release();
        d_al.release(); d_fg.release(); d_F.release(); d_sigma.release(); d_rel.release();
        d_fref.release(); d_ke.release(); d_iters.release(); d_lead.release();
        d_wint.release(); d_wext.release(); d_gp.release(); d_fdp.release();
        d_status.release(); d_queue.release(); d_counters.release(); d_naive.release();
        if (h_F) cudaFreeHost(h_F);
        h_F = nullptr;
        if (ev_F) cudaEventDestroy(ev_F);
        ev_F = nullptr;
        if (aux) cudaStreamDestroy(aux);
        aux = nullptr;
        if (ev_done) cudaEventDestroy(ev_done);
        ev_done = nullptr;
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
        if (cap) cudaStreamDestroy(cap);
        cap = nullptr;
        if (h_iters) cudaFreeHost(h_iters);
        h_iters = nullptr;
        if (h_queue) cudaFreeHost(h_queue);
        h_queue = nullptr;
        for (auto &sl : slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.d_ids) cudaFree(sl.d_ids);
            if (sl.d_cnt) cudaFree(sl.d_cnt);
            if (sl.d_F) cudaFree(sl.d_F);
            if (sl.d_out) cudaFree(sl.d_out);
            if (sl.d_it) cudaFree(sl.d_it);
            if (sl.d_st) cudaFree(sl.d_st);
            if (sl.h_ids) cudaFreeHost(sl.h_ids);
            if (sl.h_F) cudaFreeHost(sl.h_F);
            if (sl.h_out) cudaFreeHost(sl.h_out);
            if (sl.h_it) cudaFreeHost(sl.h_it);
            if (sl.h_st) cudaFreeHost(sl.h_st);
        }
        slots.clear();
        for (auto s : side) cudaStreamDestroy(s);
        for (auto e : ev) cudaEventDestroy(e);
        for (auto e : tev) cudaEventDestroy(e);
        side.clear();
        ev.clear();
        tev.clear();
    }
};

extern "C" {

void fe2_opts_default(fe2_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-8;
    o->max_iter = 10000000;
    o->dt_safety = 0.9;
    o->precision = FE2_PREC_MIXED;
    o->init = FE2_INIT_AFFINE;
    o->kinetic_energy = 0;
    o->block_threads = 0;
    o->lead_iters = -1;
    o->rebase_every = 0;
    o->lead_tol = 1e-2;
    o->stall_window = 0;
}

const char *fe2_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace {

bool finite3(const double *p) { return std::isfinite(p[0]) && std::isfinite(p[1]) && std::isfinite(p[2]); }

// Smallest cluster size (CTAs) for an RVE of n nodes in the mixed solver: a
// power of two with at most `target` nodes per CTA and room for the node
// state of the FP32 kernel without its element table (the larger of the two
// kernels' plain footprints, with slack for an uneven bisection), at most 16.
int min_parts(int n, int target, size_t smem_cap) {
    const size_t per_node = std::max(mixed_plain_node_bytes(0), mixed_plain_node_bytes(1));
    int C = 1;
    while (C < kMaxParts && ((n + C - 1) / C > target || per_node * ((n + C - 1) / C + 64) > smem_cap))
        C *= 2;
    return C;
}

// Process-wide launch tuning of the mixed solver per node-count bucket (log2
// of the node count), set by fe2_tuning_set, fe2_tuning_load or fe2_autotune;
// zero entries are automatic. Read when a batch is created.
fe2_tuning g_tuning = {};

int node_bucket(int n) {
    int b = 0;
    while (b < 31 && ((int64_t)2 << b) <= n) ++b;
    return b;  // 2^b <= n < 2^(b+1)
}

// Recursive coordinate bisection of `ids` into `parts` (a power of two) sets.
void rcb(std::vector<int> ids, int parts, const double *X, int64_t base,
         std::vector<std::vector<int>> &out) {
    if (parts == 1) {
        out.push_back(std::move(ids));
        return;
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i : ids)
        for (int c = 0; c < 3; ++c) {
            const double v = X[3 * (base + i) + c];
            lo[c] = std::min(lo[c], v);
            hi[c] = std::max(hi[c], v);
        }
    int ax = 0;
    for (int c = 1; c < 3; ++c)
        if (hi[c] - lo[c] > hi[ax] - lo[ax]) ax = c;
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) {
        const double va = X[3 * (base + a) + ax], vb = X[3 * (base + b) + ax];
        return va < vb || (va == vb && a < b);
    });
    const size_t half = ids.size() / 2;
    rcb(std::vector<int>(ids.begin(), ids.begin() + half), parts / 2, X, base, out);
    rcb(std::vector<int>(ids.begin() + half, ids.end()), parts / 2, X, base, out);
}

// Bucket RVEs into launch classes. FP64: by staged footprint (24 B/node), so
// small RVEs are not limited by the occupancy of the largest; RVEs too big for
// shared memory stage in L2 scratch. Mixed: by cluster size.
void build_classes(const std::vector<RveDesc> &rve, const std::vector<int32_t> &part_free_max,
                   size_t smem_optin, int precision, std::vector<SizeClass> &out) {
    out.clear();
    std::vector<int32_t> order(rve.size());
    std::iota(order.begin(), order.end(), 0);
    // longest-processing-time first: largest RVEs lead the queue
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return rve[x].n_free > rve[y].n_free;
    });
    const size_t cap = smem_optin - 16384;  // room for static shared memory
    if (precision == FE2_PREC_FP64) {
        // RVEs of several parts run on a cluster (one part per CTA) when its
        // position buffers fit; classes by (parts, table in shared memory).
        // FE2_FP64_CLUSTER=0 keeps every RVE on the single-CTA kernel.
        const bool clusters = env_int("FE2_FP64_CLUSTER", 1) != 0;
        auto on_cluster = [&](const RveDesc &R) {
            return clusters && R.n_parts >= 2 && fp64_cluster_smem(R.part_max, 0, 0, false, false) <= cap;
        };
        // shared-memory variant of an RVE: the element table first, then the
        // free-node state, as far as they fit
        auto variant = [&](int pm, int fm, int sm, bool &tsm, bool &ssm) {
            const bool opts[4][2] = {{true, true}, {true, false}, {false, true}, {false, false}};
            for (const auto &o : opts)
                if (fp64_cluster_smem(pm, fm, sm, o[0], o[1]) <= cap) {
                    tsm = o[0];
                    ssm = o[1];
                    return;
                }
        };
        for (int32_t p : order) {
            const RveDesc &R = rve[p];
            if (!on_cluster(R)) continue;
            bool tsm = false, ssm = false;
            variant(R.part_max, part_free_max[p], R.part_fslot_max, tsm, ssm);
            SizeClass *c = nullptr;
            for (auto &k : out)
                if (k.parts == R.n_parts && k.fp64_tsm == tsm && k.fp64_ssm == ssm &&
                    fp64_cluster_smem(std::max(k.part_max, R.part_max), std::max(k.free_max, part_free_max[p]),
                                      std::max(k.fslot_max, R.part_fslot_max), tsm, ssm) <= cap) {
                    c = &k;
                    break;
                }
            if (!c) {
                out.emplace_back();
                c = &out.back();
                c->parts = R.n_parts;
                c->fp64_cluster = true;
                c->fp64_tsm = tsm;
                c->fp64_ssm = ssm;
                c->smem_positions = 0;
            }
            c->rves.push_back(p);
            c->part_max = std::max(c->part_max, R.part_max);
            c->free_max = std::max(c->free_max, part_free_max[p]);
            c->fslot_max = std::max(c->fslot_max, R.part_fslot_max);
            c->smem_bytes = fp64_cluster_smem(c->part_max, c->free_max, c->fslot_max, c->fp64_tsm, c->fp64_ssm);
        }
        std::stable_sort(out.begin(), out.end(), [](const SizeClass &a, const SizeClass &b) {
            return a.parts > b.parts;
        });
        const size_t bounds[] = {16u << 10, 32u << 10, 56u << 10, 112u << 10, cap};
        std::vector<SizeClass> cls(6);
        cls[5].smem_positions = 0;
        for (int32_t p : order) {
            if (on_cluster(rve[p])) continue;
            const size_t need = (size_t)24 * rve[p].n_nodes;
            int c = 5;
            for (int k = 0; k < 5; ++k)
                if (need <= bounds[k] && need <= cap) { c = k; break; }
            cls[c].rves.push_back(p);
            if (c < 5) cls[c].smem_bytes = std::max(cls[c].smem_bytes, need);
        }
        for (auto &c : cls)
            if (!c.rves.empty()) out.push_back(c);
    } else {
        // A class is keyed by the cluster size and by whether each kernel keeps
        // its element table in shared memory, both decided by the RVE alone
        // (its own parts and table sizes), so an RVE runs the same code path,
        // with the same CTA size, whatever batch it is in. RVEs of one key are
        // packed first-fit into classes whose combined tables still fit.
        const size_t limit = cap;
        auto fits = [&](const SizeClass &c) {
            const bool l = !c.lead_staged || mixed_staged(1, mixed_lead_smem(c.part_max, c.free_max, c.elem_max,
                                                                             c.slot_max, limit), c.part_max);
            const bool f = !c.fp32_staged || mixed_staged(0, mixed_fp32_smem(c.part_max, c.free_max, c.elem_max,
                                                                             c.slot_max, limit), c.part_max);
            return l && f;
        };
        // first-fit decreasing: the RVEs with the largest shared-memory needs
        // open the classes, so that smaller ones fit under their maxima (the
        // queue order inside a class is restored to LPT afterwards)
        std::vector<size_t> need(rve.size(), 0);
        for (int32_t p : order)
            need[p] = mixed_fp32_smem(rve[p].part_max, part_free_max[p], rve[p].part_elem_max,
                                      rve[p].part_slot_max, (size_t)1 << 40);
        std::vector<int32_t> ffd = order;
        std::stable_sort(ffd.begin(), ffd.end(), [&](int32_t x, int32_t y) { return need[x] > need[y]; });
        std::vector<int32_t> rank(rve.size(), 0);
        for (size_t k = 0; k < order.size(); ++k) rank[order[k]] = (int32_t)k;
        for (int32_t p : ffd) {
            const RveDesc &R = rve[p];
            SizeClass one;
            one.parts = R.n_parts;
            one.part_max = R.part_max;
            one.free_max = part_free_max[p];
            one.elem_max = R.part_elem_max;
            one.slot_max = R.part_slot_max;
            one.lead_staged = mixed_staged(1, mixed_lead_smem(one.part_max, one.free_max, one.elem_max,
                                                              one.slot_max, limit), one.part_max);
            one.fp32_staged = mixed_staged(0, mixed_fp32_smem(one.part_max, one.free_max, one.elem_max,
                                                              one.slot_max, limit), one.part_max);
            const int bk = node_bucket(R.n_nodes);
            one.block_lead = g_tuning.block_lead[bk];
            one.block_fp32 = g_tuning.block_fp32[bk];
            bool placed = false;
            for (auto &c : out) {
                if (c.parts != one.parts || c.lead_staged != one.lead_staged || c.fp32_staged != one.fp32_staged ||
                    c.block_lead != one.block_lead || c.block_fp32 != one.block_fp32)
                    continue;
                SizeClass t = c;
                t.part_max = std::max(t.part_max, one.part_max);
                t.free_max = std::max(t.free_max, one.free_max);
                t.elem_max = std::max(t.elem_max, one.elem_max);
                t.slot_max = std::max(t.slot_max, one.slot_max);
                if (!fits(t)) continue;
                t.rves.push_back(p);
                c = std::move(t);
                placed = true;
                break;
            }
            if (!placed) {
                one.rves.push_back(p);
                out.push_back(std::move(one));
            }
        }
        for (auto &c : out)
            std::stable_sort(c.rves.begin(), c.rves.end(), [&](int32_t x, int32_t y) { return rank[x] < rank[y]; });
        // the class holding the largest RVEs (longest critical path) first
        std::stable_sort(out.begin(), out.end(), [](const SizeClass &a, const SizeClass &b) {
            return a.parts > b.parts;
        });
        for (auto &c : out)
            c.smem_bytes = mixed_plain_node_bytes(0) * c.part_max;
    }
    int32_t off = 0;
    for (auto &c : out) {
        c.queue_off = off;
        off += (int32_t)c.rves.size();
    }
}

int mixed_block(int requested, bool lead, bool staged);

// Dynamic shared memory of a mixed class's lead (lead = 1) or FP32 kernel:
// with the element table when the class is staged for that kernel.
size_t class_smem(const SizeClass &c, int lead, size_t limit) {
    const bool st = lead ? c.lead_staged : c.fp32_staged;
    if (!st) return mixed_plain_node_bytes(lead) * (size_t)c.part_max;
    return lead ? mixed_lead_smem(c.part_max, c.free_max, c.elem_max, c.slot_max, limit)
                : mixed_fp32_smem(c.part_max, c.free_max, c.elem_max, c.slot_max, limit);
}

// CTA size of a mixed class's kernel: the caller's request, else the tuned
// size of its RVEs' size bucket, else the default.
int class_block(const SizeClass &c, int lead, int requested) {
    const bool st = lead ? c.lead_staged : c.fp32_staged;
    const int tuned = lead ? c.block_lead : c.block_fp32;
    return mixed_block(requested ? requested : tuned, lead != 0, st);
}

// Input validation of fe2_batch_create and the inspection calls (host only).
fe2_status validate_batch(int32_t n_rve, const int64_t *node_off, const double *X,
                          const int64_t *elem_off, const int32_t *conn, const double *EA,
                          const uint8_t *fixed, const double *V0, const double *damping) {
    if (n_rve < 1) return fail(FE2_EINVAL, "n_rve must be >= 1");
    if (!node_off || !X || !elem_off || !fixed) return fail(FE2_EINVAL, "NULL input array");
    if (node_off[0] != 0 || elem_off[0] != 0) return fail(FE2_EINVAL, "offsets must start at 0");
    for (int32_t p = 0; p < n_rve; ++p) {
        if (node_off[p + 1] <= node_off[p]) return fail(FE2_EINVAL, "RVE " + std::to_string(p) + " has no nodes");
        if (node_off[p + 1] - node_off[p] > (1 << 20))
            return fail(FE2_EINVAL, "RVE " + std::to_string(p) + " has more than 2^20 nodes");
        if (elem_off[p + 1] < elem_off[p]) return fail(FE2_EINVAL, "element offsets decrease");
    }
    const int64_t N = node_off[n_rve], E = elem_off[n_rve];
    if (E > 0 && (!conn || !EA)) return fail(FE2_EINVAL, "NULL conn or EA");
    if (2 * E >= ((int64_t)1 << 31)) return fail(FE2_EINVAL, "too many elements in one batch");

    for (int64_t i = 0; i < N; ++i)
        if (!finite3(X + 3 * i)) return fail(FE2_EINVAL, "non-finite coordinate at node " + std::to_string(i));
    for (int32_t p = 0; p < n_rve; ++p) {
        if (V0 && !(V0[p] > 0.0 && std::isfinite(V0[p]))) return fail(FE2_EINVAL, "V0 must be > 0");
        if (damping && !(damping[p] >= 0.0 && std::isfinite(damping[p])))
            return fail(FE2_EINVAL, "damping must be finite and >= 0");
        const int64_t np_ = node_off[p + 1] - node_off[p];
        std::vector<std::pair<int64_t, int64_t>> keys;
        keys.reserve(elem_off[p + 1] - elem_off[p]);
        for (int64_t e = elem_off[p]; e < elem_off[p + 1]; ++e) {
            const int64_t a = conn[2 * e], c = conn[2 * e + 1];
            if (a < 0 || c < 0 || a >= np_ || c >= np_)
                return fail(FE2_EINVAL, "element " + std::to_string(e) + ": node id out of range");
            if (a == c) return fail(FE2_EINVAL, "element " + std::to_string(e) + " joins a node to itself");
            if (!(EA[e] > 0.0 && std::isfinite(EA[e])))
                return fail(FE2_EINVAL, "element " + std::to_string(e) + ": EA must be finite and > 0");
            const double *xa = X + 3 * (node_off[p] + a), *xb = X + 3 * (node_off[p] + c);
            if (xa[0] == xb[0] && xa[1] == xb[1] && xa[2] == xb[2])
                return fail(FE2_EINVAL, "element " + std::to_string(e) + " has zero length");
            keys.emplace_back(std::min(a, c), std::max(a, c));
        }
        std::sort(keys.begin(), keys.end());
        if (std::adjacent_find(keys.begin(), keys.end()) != keys.end())
            return fail(FE2_EINVAL, "RVE " + std::to_string(p) + " repeats an element");
    }
    return FE2_OK;
}

// Host-side packing of a validated batch: per RVE its parts (recursive
// coordinate bisection) and node permutation (free nodes part by part, then
// fixed nodes), its CSR rows in permuted order with the neighbour as both an
// RVE-local id and (part, index in part), and the element list; plus the
// per-RVE descriptors without device offsets filled in later.
struct HostLayout {
    std::vector<RveDesc> rve;
    std::vector<int64_t> perm_to_orig;   // permuted global -> caller global node
    std::vector<int32_t> part_free_max;  // per RVE, most free nodes in one part
    std::vector<double> X, EAcsr, ElEA;  // X as SoA [3][N]
    std::vector<int32_t> col, colp, Ela, Elb, row, part, csrEl;
    std::vector<int64_t> ElemOf, Ga, Gb;
    // FP64 cluster kernel: per part, one slot per element with an end among
    // the part's free nodes (first use in row order); per slot (element,
    // first end, second end) with ends as (part << 16 | index in part); per
    // CSR entry of a free node its slot << 1 | 1 when the node is the second
    // end; per RVE the parts' slot offsets (relative to RveDesc::slot0)
    std::vector<int32_t> fpSlot, fpCsrSlot, fpPartSlot;
};

void build_layout(int32_t n_rve, const int64_t *node_off, const double *X, const int64_t *elem_off,
                  const int32_t *conn, const double *EA, const uint8_t *fixed, const double *V0,
                  const double *damping, int target, size_t smem_cap, HostLayout &L) {
    const int64_t N = node_off[n_rve], E = elem_off[n_rve];
    L.rve.assign(n_rve, RveDesc{});
    L.perm_to_orig.assign(N, 0);
    L.part_free_max.assign(n_rve, 0);
    L.X.assign(3 * N, 0.0);
    L.EAcsr.assign(2 * E, 0.0);
    L.ElEA.assign(E, 0.0);
    L.col.assign(2 * E, 0);
    L.colp.assign(2 * E, 0);
    L.csrEl.assign(2 * E, 0);
    L.fpCsrSlot.assign(2 * E, -1);
    L.fpPartSlot.assign((size_t)n_rve * (kMaxParts + 1), 0);
    L.fpSlot.clear();
    L.Ela.assign(E, 0);
    L.Elb.assign(E, 0);
    L.ElemOf.assign(2 * E, 0);
    L.Ga.assign(E, 0);
    L.Gb.assign(E, 0);
    L.row.assign((size_t)N + n_rve, 0);
    L.part.assign((size_t)n_rve * 2 * (kMaxParts + 1), 0);
    std::vector<double> &hX = L.X, &hEAcsr = L.EAcsr, &hElEA = L.ElEA;
    std::vector<int32_t> &hcol = L.col, &hcolp = L.colp, &hEla = L.Ela, &hElb = L.Elb, &hrow = L.row,
                         &hpart = L.part;
    std::vector<int64_t> &hElemOf = L.ElemOf, &hGa = L.Ga, &hGb = L.Gb;
    int64_t csr_pos = 0;
    for (int32_t p = 0; p < n_rve; ++p) {
        const int64_t base = node_off[p];
        const int n = (int)(node_off[p + 1] - base);
        const int64_t e0 = elem_off[p], ne = elem_off[p + 1] - e0;
        std::vector<int> deg(n, 0);
        for (int64_t e = e0; e < e0 + ne; ++e) { deg[conn[2 * e]]++; deg[conn[2 * e + 1]]++; }
        std::vector<uint8_t> fx(n);
        for (int i = 0; i < n; ++i) fx[i] = (fixed[base + i] != 0) || deg[i] == 0;
        // CSR rows (caller ids), independent of the partition
        std::vector<std::vector<std::pair<int, int64_t>>> rows(n);
        for (int64_t e = e0; e < e0 + ne; ++e) {
            const int a = conn[2 * e], c = conn[2 * e + 1];
            rows[a].push_back({c, e});
            rows[c].push_back({a, e});
        }
        for (auto &row : rows) std::sort(row.begin(), row.end());
        // Parts: the smallest cluster that holds the plain state, doubled
        // (up to 16) while the FP32 kernel's element table does not fit in
        // shared memory; the autotuner may fix the count per size bucket.
        int C = min_parts(n, target, smem_cap);
        const int want = g_tuning.parts[node_bucket(n)];
        const bool forced = want >= C && want <= kMaxParts && (want & (want - 1)) == 0;
        if (forced) C = want;
        std::vector<std::vector<int>> fr, fxd;
        std::vector<int> owner(n), local(n);
        int part_max = 0, free_max = 0, elem_max = 0, slot_max = 0;
        for (;;) {
            std::vector<int> all(n);
            std::iota(all.begin(), all.end(), 0);
            std::vector<std::vector<int>> parts;
            rcb(all, C, X, base, parts);
            fr.assign(C, {});
            fxd.assign(C, {});
            for (int r = 0; r < C; ++r) {
                for (int i : parts[r]) (fx[i] ? fxd[r] : fr[r]).push_back(i);
                std::stable_sort(fr[r].begin(), fr[r].end(), [&](int x, int y) {
                    return deg[x] > deg[y] || (deg[x] == deg[y] && x < y);
                });
                std::sort(fxd[r].begin(), fxd[r].end());
                for (size_t k = 0; k < fr[r].size(); ++k) { owner[fr[r][k]] = r; local[fr[r][k]] = (int)k; }
                for (size_t k = 0; k < fxd[r].size(); ++k) {
                    owner[fxd[r][k]] = r;
                    local[fxd[r][k]] = (int)(fr[r].size() + k);
                }
            }
            // FP32 kernel tables per part: elements with an end among the part's
            // free nodes, once each (an element between two of them counted at
            // its lower local index), and row slots in slabs of 32 free nodes,
            // each 32 slots wide per entry of its longest row
            part_max = free_max = elem_max = slot_max = 0;
            for (int r = 0; r < C; ++r) {
                part_max = std::max(part_max, (int)(fr[r].size() + fxd[r].size()));
                free_max = std::max(free_max, (int)fr[r].size());
                int elems = 0, slots = 0;
                for (size_t k = 0; k < fr[r].size(); ++k) {
                    const int i = fr[r][k];
                    for (const auto &pr : rows[i]) {
                        const int j = pr.first;
                        elems += !(owner[j] == r && !fx[j] && local[j] < (int)k);
                    }
                }
                for (size_t k0 = 0; k0 < fr[r].size(); k0 += 32) {
                    int w = 0;
                    for (size_t k = k0; k < k0 + 32 && k < fr[r].size(); ++k) w = std::max(w, deg[fr[r][k]]);
                    slots += 32 * w;
                }
                elem_max = std::max(elem_max, elems);
                slot_max = std::max(slot_max, slots);
            }
            const bool staged = mixed_staged(0, mixed_fp32_smem(part_max, free_max, elem_max, slot_max, smem_cap),
                                             part_max);
            if (staged || C >= kMaxParts || forced) break;
            C *= 2;
        }
        // order: free nodes part by part (degree-sorted), then fixed part by part
        std::vector<int> order;
        order.reserve(n);
        int32_t *pf = hpart.data() + (size_t)p * 2 * (kMaxParts + 1);
        int32_t *pg = pf + (kMaxParts + 1);
        int nfree = 0;
        for (int r = 0; r < C; ++r) {
            pf[r] = nfree;
            for (int i : fr[r]) order.push_back(i);
            nfree += (int)fr[r].size();
        }
        for (int r = C; r <= kMaxParts; ++r) pf[r] = nfree;
        int nfixed = 0;
        for (int r = 0; r < C; ++r) {
            pg[r] = nfixed;
            for (int i : fxd[r]) order.push_back(i);
            nfixed += (int)fxd[r].size();
        }
        for (int r = C; r <= kMaxParts; ++r) pg[r] = nfixed;
        std::vector<int> newid(n);
        for (int k = 0; k < n; ++k) newid[order[k]] = k;
        RveDesc &R = L.rve[p];
        R.node0 = base;
        R.rp0 = base + p;
        R.csr0 = csr_pos;
        R.elem0 = e0;
        R.n_nodes = n;
        R.n_free = nfree;
        R.n_elems = (int32_t)ne;
        R.n_parts = C;
        R.dtc = 0.0;
        R.c = damping ? damping[p] : 0.002 * std::cbrt(512.0 / (double)n);
        R.V0 = V0 ? V0[p] : 1.0;
        R.part_max = part_max;
        R.part_free_max = free_max;
        R.part_elem_max = elem_max;
        R.part_slot_max = slot_max;
        L.part_free_max[p] = free_max;
        int32_t pos = 0;
        for (int k = 0; k < n; ++k) {
            const int orig = order[k];
            L.perm_to_orig[base + k] = base + orig;
            for (int r = 0; r < 3; ++r) hX[r * N + base + k] = X[3 * (base + orig) + r];
            auto &row = rows[orig];
            std::sort(row.begin(), row.end());
            hrow[R.rp0 + k] = pos;
            for (auto &pr : row) {
                hcol[csr_pos + pos] = newid[pr.first];
                hcolp[csr_pos + pos] = (owner[pr.first] << 16) | local[pr.first];
                hElemOf[csr_pos + pos] = pr.second;
                L.csrEl[csr_pos + pos] = (int32_t)(((pr.second - e0) << 1) | (conn[2 * pr.second + 1] == orig ? 1 : 0));
                hEAcsr[csr_pos + pos] = EA[pr.second];
                ++pos;
            }
        }
        hrow[R.rp0 + n] = pos;
        // FP64 cluster slot tables (see HostLayout)
        {
            R.slot0 = (int64_t)(L.fpSlot.size() / 4);
            int32_t *ps = L.fpPartSlot.data() + (size_t)p * (kMaxParts + 1);
            std::vector<int32_t> slot_of(ne, -1);
            int32_t ns = 0, fslot_max = 0;
            for (int r = 0; r < C; ++r) {
                ps[r] = ns;
                const int32_t first = ns;
                for (int k = pf[r]; k < pf[r + 1]; ++k) {
                    for (int32_t q = hrow[R.rp0 + k]; q < hrow[R.rp0 + k + 1]; ++q) {
                        const int32_t w = L.csrEl[csr_pos + q];
                        const int32_t e = w >> 1;
                        if (slot_of[e] < first) {  // not yet a slot of this part
                            slot_of[e] = ns++;
                            const int a = conn[2 * (e0 + e)], c2 = conn[2 * (e0 + e) + 1];
                            L.fpSlot.push_back(e);
                            L.fpSlot.push_back((owner[a] << 16) | local[a]);
                            L.fpSlot.push_back((owner[c2] << 16) | local[c2]);
                            L.fpSlot.push_back(0);
                        }
                        L.fpCsrSlot[csr_pos + q] = ((slot_of[e] - first) << 1) | (w & 1);
                    }
                }
                fslot_max = std::max(fslot_max, ns - first);
            }
            for (int r = C; r <= kMaxParts; ++r) ps[r] = ns;
            R.part_fslot_max = fslot_max;
        }
        csr_pos += pos;
        for (int64_t e = e0; e < e0 + ne; ++e) {
            // the caller's orientation (a, b) is kept for lengths and the stress sum
            hEla[e] = newid[conn[2 * e]];
            hElb[e] = newid[conn[2 * e + 1]];
            hGa[e] = base + newid[conn[2 * e]];
            hGb[e] = base + newid[conn[2 * e + 1]];
            hElEA[e] = EA[e];
        }
    }

}

}  // namespace

extern "C" fe2_status fe2_batch_create(int32_t n_rve, const int64_t *node_off, const double *X,
                                       const int64_t *elem_off, const int32_t *conn,
                                       const double *EA, const uint8_t *fixed, const double *V0,
                                       const double *damping, void *stream, fe2_batch **out) {
    if (!out) return fail(FE2_EINVAL, "out is NULL");
    *out = nullptr;
    {
        const fe2_status v = validate_batch(n_rve, node_off, X, elem_off, conn, EA, fixed, V0, damping);
        if (v != FE2_OK) return v;
    }
    const int64_t N = node_off[n_rve], E = elem_off[n_rve];

    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    if (prop.major != 10 || prop.minor != 3)
        return fail(FE2_ENODEV, std::string("need an sm_103 GPU, found ") + prop.name);

    fe2_batch *b = new fe2_batch();
    b->n_rve = n_rve;
    b->n_nodes = N;
    b->n_elems = E;
    b->n_csr = 2 * E;
    b->device = dev;
    b->sm_count = prop.multiProcessorCount;
    b->smem_optin = prop.sharedMemPerBlockOptin;
    b->rve.resize(n_rve);
    b->perm_to_orig.resize(N);
    b->part_free_max.resize(n_rve);
    const int target = std::max(64, env_int("FE2_NODES_PER_CTA", 1024));
    const size_t smem_cap = b->smem_optin - 16384;

    // ---- packing: parts, permutation, CSR rows, element list ----
    HostLayout L;
    build_layout(n_rve, node_off, X, elem_off, conn, EA, fixed, V0, damping, target, smem_cap, L);
    b->rve = L.rve;
    b->perm_to_orig = L.perm_to_orig;
    b->part_free_max = L.part_free_max;
    std::vector<double> &hX = L.X, &hEAcsr = L.EAcsr, &hElEA = L.ElEA;
    std::vector<int32_t> &hcol = L.col, &hcolp = L.colp, &hEla = L.Ela, &hElb = L.Elb, &hrow = L.row,
                         &hpart = L.part;
    std::vector<int64_t> &hElemOf = L.ElemOf, &hGa = L.Ga, &hGb = L.Gb;

    // ---- device allocation and upload ----
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fe2_status rc = FE2_OK;
    auto A = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && rc == FE2_OK) {
            rc = e == cudaErrorMemoryAllocation ? FE2_ENOMEM : FE2_ECUDA;
            g_err = std::string(what) + ": " + cudaGetErrorString(e);
        }
    };
    DevBuf<int64_t> d_elemof, d_ga, d_gb;
    A(b->d_rve.alloc(n_rve), "rve");
    A(b->d_X.alloc(3 * N), "X");
    A(b->d_Xh.alloc(3 * N), "Xh");
    A(b->d_Xl.alloc(3 * N), "Xl");
    A(b->d_mass.alloc(N), "mass");
    A(b->d_imh.alloc(N), "imh");
    A(b->d_iml.alloc(N), "iml");
    A(b->d_EA_csr.alloc(2 * E), "EA_csr");
    A(b->d_L_csr.alloc(2 * E), "L_csr");
    A(b->d_eaf.alloc(2 * E), "eaf");
    A(b->d_eaf_lo.alloc(2 * E), "eaf_lo");
    A(b->d_dh.alloc(2 * E), "dh");
    A(b->d_dl.alloc(2 * E), "dl");
    A(b->d_col.alloc(2 * E), "col");
    A(b->d_col_part.alloc(2 * E), "col_part");
    A(b->d_csr_el.alloc(2 * E), "csr_el");
    const size_t n_fslots = L.fpSlot.size() / 4;
    A(b->d_fp_slot.alloc(std::max<size_t>(1, n_fslots)), "fp_slot");
    A(b->d_fp_csr_slot.alloc(2 * E), "fp_csr_slot");
    A(b->d_fp_part_slot.alloc(L.fpPartSlot.size()), "fp_part_slot");
    A(b->d_ualt.alloc(3 * N), "ualt");
    A(b->d_fpt.alloc(3 * std::max<size_t>(1, n_fslots)), "fpt");
    A(b->d_tf.alloc(3 * E), "tf");
    A(b->d_sv.alloc(N), "sv");
    A(b->d_sa.alloc(N), "sa");
    A(b->d_rowptr.alloc(N + n_rve), "rowptr");
    A(b->d_part_off.alloc(hpart.size()), "part_off");
    A(b->d_el_a.alloc(E), "el_a");
    A(b->d_el_b.alloc(E), "el_b");
    A(b->d_el_EA.alloc(E), "el_EA");
    A(b->d_el_L.alloc(E), "el_L");
    A(b->d_u.alloc(3 * N), "u");
    A(b->d_v.alloc(3 * N), "v");
    A(b->d_a.alloc(3 * N), "a");
    A(b->d_xg.alloc(3 * N), "xg");
    A(b->d_uh.alloc(3 * N), "uh");
    A(b->d_ul.alloc(3 * N), "ul");
    A(b->d_vh.alloc(3 * N), "vh");
    A(b->d_vl.alloc(3 * N), "vl");
    A(b->d_ah.alloc(3 * N), "ah");
    A(b->d_al.alloc(3 * N), "al");
    A(b->d_fg.alloc(3 * N), "fg");
    A(b->d_F.alloc(9 * (size_t)n_rve), "F");
    A(b->d_sigma.alloc(9 * (size_t)n_rve), "sigma");
    A(b->d_rel.alloc(n_rve), "rel");
    A(b->d_fref.alloc(n_rve), "fref");
    A(b->d_ke.alloc(n_rve), "ke");
    A(b->d_wint.alloc(n_rve), "wint");
    A(b->d_wext.alloc(n_rve), "wext");
    A(b->d_gp.alloc(3 * N), "gp");
    A(b->d_fdp.alloc(3 * N), "fdp");
    A(b->d_iters.alloc(n_rve), "iters");
    A(b->d_lead.alloc(n_rve), "lead");
    A(b->d_status.alloc(n_rve), "status");
    A(b->d_queue.alloc(2 * (size_t)n_rve), "queue");
    A(b->d_counters.alloc(kCountersPerClass * (size_t)n_rve + 16), "counters");
    A(d_elemof.alloc(2 * E), "elemof");
    A(d_ga.alloc(E), "ga");
    A(d_gb.alloc(E), "gb");
    auto H2D = [&](void *dst, const void *src, size_t bytes, const char *what) {
        if (bytes && rc == FE2_OK) A(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st), what);
    };
    H2D(b->d_rve.p, b->rve.data(), sizeof(RveDesc) * n_rve, "rve");
    H2D(b->d_X.p, hX.data(), sizeof(double) * 3 * N, "X");
    H2D(b->d_EA_csr.p, hEAcsr.data(), sizeof(double) * 2 * E, "EA_csr");
    H2D(b->d_col.p, hcol.data(), sizeof(int32_t) * 2 * E, "col");
    H2D(b->d_col_part.p, hcolp.data(), sizeof(int32_t) * 2 * E, "col_part");
    H2D(b->d_csr_el.p, L.csrEl.data(), sizeof(int32_t) * 2 * E, "csr_el");
    if (n_fslots) H2D(b->d_fp_slot.p, L.fpSlot.data(), sizeof(int4) * n_fslots, "fp_slot");
    H2D(b->d_fp_csr_slot.p, L.fpCsrSlot.data(), sizeof(int32_t) * 2 * E, "fp_csr_slot");
    H2D(b->d_fp_part_slot.p, L.fpPartSlot.data(), sizeof(int32_t) * L.fpPartSlot.size(), "fp_part_slot");
    H2D(b->d_rowptr.p, hrow.data(), sizeof(int32_t) * (N + n_rve), "rowptr");
    H2D(b->d_part_off.p, hpart.data(), sizeof(int32_t) * hpart.size(), "part_off");
    H2D(b->d_el_a.p, hEla.data(), sizeof(int32_t) * E, "el_a");
    H2D(b->d_el_b.p, hElb.data(), sizeof(int32_t) * E, "el_b");
    H2D(b->d_el_EA.p, hElEA.data(), sizeof(double) * E, "el_EA");
    H2D(d_elemof.p, hElemOf.data(), sizeof(int64_t) * 2 * E, "elemof");
    H2D(d_ga.p, hGa.data(), sizeof(int64_t) * E, "ga");
    H2D(d_gb.p, hGb.data(), sizeof(int64_t) * E, "gb");
    if (rc == FE2_OK) A(cudaMemsetAsync(b->d_u.p, 0, sizeof(double) * 3 * N, st), "u zero");
    if (rc == FE2_OK) {
        const int e = launch_setup(n_rve, E, 2 * E, b->d_rve.p, d_ga.p, d_gb.p, b->d_X.p,
                                   b->d_X.p + N, b->d_X.p + 2 * N, d_elemof.p, b->d_EA_csr.p,
                                   b->d_el_EA.p, b->d_rowptr.p, b->d_el_L.p, b->d_L_csr.p,
                                   b->d_eaf.p, b->d_eaf_lo.p, b->d_mass.p, b->d_imh.p,
                                   b->d_iml.p, b->d_Xh.p, b->d_Xl.p, b->d_col.p, b->d_dh.p,
                                   b->d_dl.p, st);
        A((cudaError_t)e, "setup kernels");
    }
    if (rc == FE2_OK)
        A(cudaMemcpyAsync(b->rve.data(), b->d_rve.p, sizeof(RveDesc) * n_rve, cudaMemcpyDeviceToHost, st),
          "rve readback");
    if (rc == FE2_OK) A(cudaStreamSynchronize(st), "create sync");
    d_elemof.release(); d_ga.release(); d_gb.release();
    if (rc == FE2_OK) {
        build_classes(b->rve, b->part_free_max, b->smem_optin, FE2_PREC_FP64, b->classes_fp64);
        build_classes(b->rve, b->part_free_max, b->smem_optin, FE2_PREC_MIXED, b->classes_mixed);
        // work queues: per class, RVE ids in scheduling order (FP64, then mixed)
        std::vector<int32_t> q(2 * (size_t)n_rve);
        for (auto &c : b->classes_fp64) std::copy(c.rves.begin(), c.rves.end(), q.begin() + c.queue_off);
        for (auto &c : b->classes_mixed)
            std::copy(c.rves.begin(), c.rves.end(), q.begin() + n_rve + c.queue_off);
        A(cudaMemcpy(b->d_queue.p, q.data(), sizeof(int32_t) * 2 * n_rve, cudaMemcpyHostToDevice), "queue");
        A(cudaMallocHost(&b->h_F, sizeof(double) * 9 * n_rve), "pinned F");
        A(cudaEventCreateWithFlags(&b->ev_F, cudaEventDisableTiming), "F event");
        A(cudaMallocHost(&b->h_iters, sizeof(int64_t) * n_rve), "pinned iters");
        A(cudaMallocHost(&b->h_queue, sizeof(int32_t) * 2 * n_rve), "pinned queue");
        A(cudaStreamCreateWithFlags(&b->aux, cudaStreamNonBlocking), "aux stream");
        A(cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming), "done event");
        A(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking), "capture stream");
    }
    // one stream per launch class (at least 8), so that classes never queue
    // behind each other
    const size_t n_side = std::max<size_t>(8, std::max(b->classes_fp64.size(), b->classes_mixed.size()));
    for (size_t k = 0; k < n_side && rc == FE2_OK; ++k) {
        cudaStream_t s;
        A(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
        if (rc == FE2_OK) b->side.push_back(s);
    }
    if (rc == FE2_OK) {
        b->class_of_fp64.assign(n_rve, 0);
        b->class_of_mixed.assign(n_rve, 0);
        for (size_t k = 0; k < b->classes_fp64.size(); ++k)
            for (int32_t p : b->classes_fp64[k].rves) b->class_of_fp64[p] = (int32_t)k;
        for (size_t k = 0; k < b->classes_mixed.size(); ++k)
            for (int32_t p : b->classes_mixed[k].rves) b->class_of_mixed[p] = (int32_t)k;
        b->in_flight.assign(n_rve, 0);
        b->slots.resize(kServeSlots);
        for (auto &sl : b->slots) {
            A(cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking), "slot stream");
            A(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming), "slot event");
            A(cudaMalloc(&sl.d_ids, sizeof(int32_t) * 2 * n_rve), "slot ids");
            A(cudaMalloc(&sl.d_cnt, sizeof(int32_t) * (kCountersPerClass * (size_t)n_rve + 16)), "slot counters");
            A(cudaMalloc(&sl.d_F, sizeof(double) * 9 * n_rve), "slot F");
            A(cudaMalloc(&sl.d_out, sizeof(double) * 10 * n_rve), "slot out");
            A(cudaMalloc(&sl.d_it, sizeof(int64_t) * n_rve), "slot iters");
            A(cudaMalloc(&sl.d_st, sizeof(int32_t) * n_rve), "slot status");
            A(cudaMallocHost(&sl.h_ids, sizeof(int32_t) * 2 * n_rve), "slot pinned ids");
            A(cudaMallocHost(&sl.h_F, sizeof(double) * 9 * n_rve), "slot pinned F");
            A(cudaMallocHost(&sl.h_out, sizeof(double) * 10 * n_rve), "slot pinned out");
            A(cudaMallocHost(&sl.h_it, sizeof(int64_t) * n_rve), "slot pinned iters");
            A(cudaMallocHost(&sl.h_st, sizeof(int32_t) * n_rve), "slot pinned status");
            if (rc != FE2_OK) break;
        }
    }
    const size_t ncls = std::max(b->classes_fp64.size(), b->classes_mixed.size());
    for (size_t k = 0; k < ncls + 2 && rc == FE2_OK; ++k) {
        cudaEvent_t e;
        A(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        if (rc == FE2_OK) b->ev.push_back(e);
    }
    for (size_t k = 0; k < 6 * ncls + 8 && rc == FE2_OK; ++k) {
        cudaEvent_t e;
        A(cudaEventCreate(&e), "timing event");
        if (rc == FE2_OK) b->tev.push_back(e);
    }
    if (rc != FE2_OK) {
        b->release();
        delete b;
        return rc;
    }
    *out = b;
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_layout(int32_t n_rve, const int64_t *node_off, const double *X,
                                       const int64_t *elem_off, const int32_t *conn,
                                       const double *EA, const uint8_t *fixed, int64_t smem_optin,
                                       int32_t nodes_per_cta, int32_t *parts, int64_t *perm,
                                       int32_t *rowptr, int32_t *col, int32_t *col_part,
                                       int32_t *part_off) {
    const fe2_status v = validate_batch(n_rve, node_off, X, elem_off, conn, EA, fixed, nullptr, nullptr);
    if (v != FE2_OK) return v;
    if (smem_optin <= 16384) return fail(FE2_EINVAL, "smem_optin must exceed 16384 bytes");
    const int target = std::max(64, nodes_per_cta > 0 ? nodes_per_cta : env_int("FE2_NODES_PER_CTA", 1024));
    HostLayout L;
    build_layout(n_rve, node_off, X, elem_off, conn, EA, fixed, nullptr, nullptr, target,
                 (size_t)smem_optin - 16384, L);
    if (parts)
        for (int32_t p = 0; p < n_rve; ++p) parts[p] = L.rve[p].n_parts;
    if (perm) std::copy(L.perm_to_orig.begin(), L.perm_to_orig.end(), perm);
    if (rowptr) std::copy(L.row.begin(), L.row.end(), rowptr);
    if (col) std::copy(L.col.begin(), L.col.end(), col);
    if (col_part) std::copy(L.colp.begin(), L.colp.end(), col_part);
    if (part_off) std::copy(L.part.begin(), L.part.end(), part_off);
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_fp64_slots(int32_t n_rve, const int64_t *node_off, const double *X,
                                           const int64_t *elem_off, const int32_t *conn, const double *EA,
                                           const uint8_t *fixed, int64_t smem_optin, int32_t nodes_per_cta,
                                           int64_t cap, int64_t *n_slots, int64_t *slot0, int32_t *part_slot,
                                           int32_t *slot, int32_t *csr_slot) {
    const fe2_status v = validate_batch(n_rve, node_off, X, elem_off, conn, EA, fixed, nullptr, nullptr);
    if (v != FE2_OK) return v;
    if (smem_optin <= 16384) return fail(FE2_EINVAL, "smem_optin must exceed 16384 bytes");
    const int target = std::max(64, nodes_per_cta > 0 ? nodes_per_cta : env_int("FE2_NODES_PER_CTA", 1024));
    HostLayout L;
    build_layout(n_rve, node_off, X, elem_off, conn, EA, fixed, nullptr, nullptr, target,
                 (size_t)smem_optin - 16384, L);
    const int64_t ns = (int64_t)(L.fpSlot.size() / 4);
    if (n_slots) *n_slots = ns;
    if (slot0)
        for (int32_t p = 0; p < n_rve; ++p) slot0[p] = L.rve[p].slot0;
    if (part_slot) std::copy(L.fpPartSlot.begin(), L.fpPartSlot.end(), part_slot);
    if (slot) std::copy(L.fpSlot.begin(), L.fpSlot.begin() + 4 * std::min(ns, std::max<int64_t>(cap, 0)), slot);
    if (csr_slot) std::copy(L.fpCsrSlot.begin(), L.fpCsrSlot.end(), csr_slot);
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_plan(int32_t n_rve, const int64_t *node_off, const double *X,
                                     const int64_t *elem_off, const int32_t *conn, const double *EA,
                                     const uint8_t *fixed, int64_t smem_optin, int32_t nodes_per_cta,
                                     int32_t max_classes, int32_t *n_classes, int32_t *rve_class,
                                     int32_t *class_parts, int32_t *class_rves, int64_t *smem,
                                     int32_t *staged, int32_t *block) {
    const fe2_status v = validate_batch(n_rve, node_off, X, elem_off, conn, EA, fixed, nullptr, nullptr);
    if (v != FE2_OK) return v;
    if (smem_optin <= 16384) return fail(FE2_EINVAL, "smem_optin must exceed 16384 bytes");
    const int target = std::max(64, nodes_per_cta > 0 ? nodes_per_cta : env_int("FE2_NODES_PER_CTA", 1024));
    HostLayout L;
    build_layout(n_rve, node_off, X, elem_off, conn, EA, fixed, nullptr, nullptr, target,
                 (size_t)smem_optin - 16384, L);
    std::vector<SizeClass> cls;
    build_classes(L.rve, L.part_free_max, (size_t)smem_optin, FE2_PREC_MIXED, cls);
    if (n_classes) *n_classes = (int32_t)cls.size();
    const size_t limit = (size_t)smem_optin - 16384;  // as in launch_class
    for (size_t k = 0; k < cls.size(); ++k) {
        const SizeClass &c = cls[k];
        if (rve_class)
            for (int32_t p : c.rves) rve_class[p] = (int32_t)k;
        if ((int32_t)k >= max_classes) continue;
        if (class_parts) class_parts[k] = c.parts;
        if (class_rves) class_rves[k] = (int32_t)c.rves.size();
        for (int lead = 1; lead >= 0; --lead) {
            const size_t sm = class_smem(c, lead, limit);
            const bool st = lead ? c.lead_staged : c.fp32_staged;
            const size_t at = 2 * k + (lead ? 0 : 1);
            if (smem) smem[at] = (int64_t)sm;
            if (staged) staged[at] = st ? 1 : 0;
            if (block) block[at] = class_block(c, lead, 0);
        }
    }
    return FE2_OK;
}

namespace {

fe2_status check_opts(const fe2_opts &o) {
    if (!(o.tol >= 0.0) || !std::isfinite(o.tol)) return fail(FE2_EINVAL, "tol must be finite and >= 0");
    if (o.max_iter < 1) return fail(FE2_EINVAL, "max_iter must be >= 1");
    if (!(o.dt_safety > 0.0 && o.dt_safety <= 1.0)) return fail(FE2_EINVAL, "dt_safety must be in (0, 1]");
    if (o.precision != FE2_PREC_FP64 && o.precision != FE2_PREC_MIXED)
        return fail(FE2_EINVAL, "unknown precision");
    if (o.init < 0 || o.init > 2) return fail(FE2_EINVAL, "unknown init");
    if (o.block_threads != 0 && (o.block_threads < 64 || o.block_threads > 512 || o.block_threads % 32))
        return fail(FE2_EINVAL, "block_threads must be 0 or a multiple of 32 in [64, 512]");
    if (!(o.lead_tol >= 0.0) || !std::isfinite(o.lead_tol)) return fail(FE2_EINVAL, "lead_tol must be finite and >= 0");
    if (o.launch != 0 && o.launch != 1) return fail(FE2_EINVAL, "launch must be 0 (graph) or 1 (stream)");
    if (o.kinetic_energy < 0 || o.kinetic_energy > 2) return fail(FE2_EINVAL, "kinetic_energy must be 0, 1 or 2");
    if (o.kinetic_energy == 2 && o.precision != FE2_PREC_FP64)
        return fail(FE2_EINVAL, "the energy-balance work terms (kinetic_energy = 2) need FE2_PREC_FP64");
    return FE2_OK;
}

// CTA size of a mixed launch: 512 threads, except the lead kernel without its
// element table (256: two CTAs per SM, its registers allow no more). The size
// is a function of the RVE (its bucket's tuning) and never of the batch, which
// keeps every RVE's result independent of which other RVEs share its launch
// (partial sums follow the thread mapping).
int mixed_block(int requested, bool lead, bool staged) {
    const int cap = lead && !staged ? 256 : 512;
    return requested ? std::min(requested, cap) : cap;
}

// Longest-processing-time order from measured cost: once a solve has
// finished, its iteration counts (times free nodes) reorder every class's
// queue so that the slowest RVEs of the next solve start first. Results do not
// depend on the order; only the tail of the launch does.
fe2_status reorder_queues(fe2_batch *b) {
    if (!b->solved || cudaEventQuery(b->ev_done) != cudaSuccess) {
        cudaGetLastError();  // clear a cudaErrorNotReady
        return FE2_OK;
    }
    const int32_t P = b->n_rve;
    CUDA_TRY(cudaMemcpyAsync(b->h_iters, b->d_iters.p, sizeof(int64_t) * P, cudaMemcpyDeviceToHost, b->aux));
    CUDA_TRY(cudaStreamSynchronize(b->aux));
    auto cost = [&](int32_t p) { return (double)std::max<int64_t>(1, b->h_iters[p]) * (b->rve[p].n_free + 1); };
    for (int which = 0; which < 2; ++which) {
        auto &classes = which == 0 ? b->classes_fp64 : b->classes_mixed;
        for (auto &c : classes) {
            std::stable_sort(c.rves.begin(), c.rves.end(), [&](int32_t x, int32_t y) { return cost(x) > cost(y); });
            std::copy(c.rves.begin(), c.rves.end(), b->h_queue + which * P + c.queue_off);
        }
    }
    CUDA_TRY(cudaMemcpyAsync(b->d_queue.p, b->h_queue, sizeof(int32_t) * 2 * P, cudaMemcpyHostToDevice, b->aux));
    CUDA_TRY(cudaStreamSynchronize(b->aux));
    return FE2_OK;
}

// Launch the solver kernels of one class on `s` for `nq` queued RVEs. Timing
// events (tev) are recorded only when `timed` is non-null.
int resident_of(fe2_batch *b, int kind, int parts, int block, size_t smem, int part_cap) {
    const auto key = std::make_tuple(kind, parts, block, smem, part_cap);
    auto it = b->occ.find(key);
    if (it != b->occ.end()) return it->second;
    // kind: 0/1 mixed FP32/lead, 2 FP64 single CTA (parts = positions staged)
    const int r = kind == 2 ? occupancy_dr_fp64(parts, block, smem)
                            : occupancy_dr_mixed(kind, parts, block, smem, part_cap);
    b->occ[key] = r;
    return r;
}

// Resident clusters of an FP64 cluster class (cached like resident_of; the
// key's kind 3 + 2 tsm + ssm and the smem size identify the variant).
int resident_fp64_cluster(fe2_batch *b, const SizeClass &c, int block) {
    const auto key = std::make_tuple(3 + 2 * (int)c.fp64_tsm + (int)c.fp64_ssm, c.parts, block, c.smem_bytes,
                                     c.part_max);
    auto it = b->occ.find(key);
    if (it != b->occ.end()) return it->second;
    const int r = occupancy_dr_fp64_cluster(c.parts, block, c.part_max, c.free_max, c.fslot_max, c.fp64_tsm,
                                            c.fp64_ssm);
    b->occ[key] = r;
    return r;
}

// Timing event around a launch: recorded as a graph node while capturing.
cudaError_t record_timing(cudaEvent_t e, cudaStream_t s, bool capturing) {
    return capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

fe2_status launch_class(fe2_batch *b, const fe2_opts &o, const SizeClass &c, SolveParams P,
                        const int32_t *queue, int nq, int32_t *counters, cudaStream_t s, int *timed,
                        int *launches, bool capturing = false) {
    const bool fp64 = o.precision == FE2_PREC_FP64;
    const DevMesh M = b->mesh();
    const DevState S = b->state();
    const DevResults R = b->results();
    P.queue = queue;
    P.queue_len = nq;
    P.counter = counters;
    P.smem_positions = c.smem_positions;
    if (fp64 && c.fp64_cluster) {
        const int block = o.block_threads ? o.block_threads : 512;
        const int resident = resident_fp64_cluster(b, c, block);
        if (resident < 1)
            return fail(FE2_ECUDA, "no FP64 cluster of " + std::to_string(c.parts) + " CTAs fits");
        if (timed) {
            if (*timed + 2 > (int)b->tev.size()) return fail(FE2_ECUDA, "too many launch classes");
            CUDA_TRY(record_timing(b->tev[*timed], s, capturing));
        }
        const int e = launch_dr_fp64_cluster(M, S, R, P, std::min(nq, resident), c.parts, block, c.part_max,
                                             c.free_max, c.fslot_max, c.fp64_tsm, c.fp64_ssm, s);
        if (e != 0) return fail(FE2_ECUDA, std::string("launch: ") + cudaGetErrorString((cudaError_t)e));
        if (timed) {
            CUDA_TRY(record_timing(b->tev[*timed + 1], s, capturing));
            *timed += 2;
        }
        ++*launches;
    } else if (fp64) {
        const int block = o.block_threads ? o.block_threads : 512;
        const size_t smem = c.smem_positions ? c.smem_bytes : 0;
        const int per_sm = std::max(1, resident_of(b, 2, c.smem_positions, block, smem, 0));
        const int grid = std::max(1, std::min<int>(nq, per_sm * b->sm_count));
        if (timed) {
            if (*timed + 2 > (int)b->tev.size()) return fail(FE2_ECUDA, "too many launch classes");
            CUDA_TRY(record_timing(b->tev[*timed], s, capturing));
        }
        const int e = launch_dr_fp64(M, S, R, P, grid, block, smem, s);
        if (e != 0) return fail(FE2_ECUDA, std::string("launch: ") + cudaGetErrorString((cudaError_t)e));
        if (timed) {
            CUDA_TRY(record_timing(b->tev[*timed + 1], s, capturing));
            *timed += 2;
        }
        ++*launches;
    } else {
        // the double-float lead, the FP32 phase, and the double-float resume
        // of RVEs whose FP32 phase stalled (a lead launch that skips the rest)
        for (int step = 0; step < 3; ++step) {
            const int lead = step == 1 ? 0 : 1;
            P.resume = step == 2 ? 1 : 0;
            const size_t limit = b->smem_optin - 16384;
            const size_t smem = class_smem(c, lead, limit);
            const int block = class_block(c, lead, o.block_threads);
            const int resident = resident_of(b, lead, c.parts, block, smem, c.part_max);
            if (resident < 1)
                return fail(FE2_ECUDA, "no cluster of " + std::to_string(c.parts) + " CTAs with " +
                                           std::to_string(smem) + " B shared memory fits");
            if (timed) {
                if (*timed + 2 > (int)b->tev.size()) return fail(FE2_ECUDA, "too many launch classes");
                CUDA_TRY(record_timing(b->tev[*timed], s, capturing));
            }
            const int e = launch_dr_mixed(M, S, R, P, lead, std::min(nq, resident), c.parts, block, smem,
                                          c.part_max, c.free_max, c.elem_max, c.slot_max, s);
            if (e != 0) return fail(FE2_ECUDA, std::string("launch: ") + cudaGetErrorString((cudaError_t)e));
            if (timed) {
                CUDA_TRY(record_timing(b->tev[*timed + 1], s, capturing));
                *timed += 2;
            }
            ++*launches;
        }
    }
    return FE2_OK;
}

SolveParams make_params(fe2_batch *b, const fe2_opts &o) {
    SolveParams P = {};
    P.F = b->d_F.p;
    P.tol = o.tol;
    P.max_iter = o.max_iter;
    P.alpha = o.dt_safety;
    P.init = o.init;
    P.want_ke = o.kinetic_energy;
    P.lead_iters = o.lead_iters;
    P.lead_tol = o.lead_tol;
    P.rebase_every = o.rebase_every;
    P.stall_window = o.stall_window == 0 ? 1000000 : (o.stall_window < 0 ? 0 : o.stall_window);
    P.resume = 0;
    return P;
}

// Serving submissions and batched solves share the per-RVE state (F, u,
// results). A batched call orders its stream after every submission still in
// flight (device-side wait), and a host readback waits for them; a submission
// waits for the last batched solve (fe2_batch_submit).
fe2_status after_slots(fe2_batch *b, cudaStream_t st) {
    for (auto &sl : b->slots)
        if (sl.busy) CUDA_TRY(cudaStreamWaitEvent(st, sl.done, 0));
    return FE2_OK;
}
fe2_status wait_slots(fe2_batch *b) {
    for (auto &sl : b->slots)
        if (sl.busy) CUDA_TRY(cudaEventSynchronize(sl.done));
    return FE2_OK;
}

// The launches of one batched solve, issued on `st`: reset the work-queue
// heads, fork one stream per class, launch each class's persistent kernels,
// join back on `st`.
fe2_status record_solve(fe2_batch *b, const fe2_opts &o, cudaStream_t st, bool capturing, int *launches,
                        int *timed) {
    const bool fp64 = o.precision == FE2_PREC_FP64;
    auto &classes = fp64 ? b->classes_fp64 : b->classes_mixed;
    CUDA_TRY(cudaMemsetAsync(b->d_counters.p, 0, sizeof(int32_t) * kCountersPerClass * classes.size(), st));
    const SolveParams P = make_params(b, o);
    CUDA_TRY(cudaEventRecord(b->ev[0], st));
    for (size_t k = 0; k < classes.size(); ++k) {
        const SizeClass &c = classes[k];
        cudaStream_t s = b->side[k % b->side.size()];
        CUDA_TRY(cudaStreamWaitEvent(s, b->ev[0], 0));
        const fe2_status r = launch_class(b, o, c, P, b->d_queue.p + (fp64 ? 0 : b->n_rve) + c.queue_off,
                                          (int)c.rves.size(), b->d_counters.p + kCountersPerClass * k, s, timed, launches,
                                          capturing);
        if (r != FE2_OK) return r;
        CUDA_TRY(cudaEventRecord(b->ev[1 + k], s));
        CUDA_TRY(cudaStreamWaitEvent(st, b->ev[1 + k], 0));
    }
    return FE2_OK;
}

// Launch shapes (resident counts, kernel attributes) of every class, queried
// before a capture so that the capture records launches only.
fe2_status warm_shapes(fe2_batch *b, const fe2_opts &o) {
    const bool fp64 = o.precision == FE2_PREC_FP64;
    const size_t limit = b->smem_optin - 16384;
    for (const SizeClass &c : fp64 ? b->classes_fp64 : b->classes_mixed) {
        if (fp64 && c.fp64_cluster) {
            const int block = o.block_threads ? o.block_threads : 512;
            if (resident_fp64_cluster(b, c, block) < 1)
                return fail(FE2_ECUDA, "no FP64 cluster of " + std::to_string(c.parts) + " CTAs fits");
            continue;
        }
        if (fp64) {
            const int block = o.block_threads ? o.block_threads : 512;
            resident_of(b, 2, c.smem_positions, block, c.smem_positions ? c.smem_bytes : 0, 0);
            continue;
        }
        for (int lead = 1; lead >= 0; --lead) {
            const size_t smem = class_smem(c, lead, limit);
            if (smem > limit) {
                int32_t big = c.rves.front();
                for (int32_t p : c.rves) if (b->rve[p].n_nodes > b->rve[big].n_nodes) big = p;
                return fail(FE2_EINVAL, "RVE " + std::to_string(big) + " (" +
                                            std::to_string(b->rve[big].n_nodes) +
                                            " nodes) exceeds the mixed solver's shared memory; use FE2_PREC_FP64");
            }
            if (resident_of(b, lead, c.parts, class_block(c, lead, o.block_threads), smem, c.part_max) < 1)
                return fail(FE2_ECUDA, "no cluster of " + std::to_string(c.parts) + " CTAs with " +
                                           std::to_string(smem) + " B shared memory fits");
        }
    }
    return FE2_OK;
}

bool same_solve_opts(const fe2_opts &a, const fe2_opts &b) {
    return a.tol == b.tol && a.max_iter == b.max_iter && a.dt_safety == b.dt_safety &&
           a.precision == b.precision && a.init == b.init && a.kinetic_energy == b.kinetic_energy &&
           a.block_threads == b.block_threads && a.lead_iters == b.lead_iters &&
           a.rebase_every == b.rebase_every && a.lead_tol == b.lead_tol && a.stall_window == b.stall_window;
}

fe2_status launch_solve(fe2_batch *b, const fe2_opts &o, cudaStream_t st) {
    {
        const fe2_status r = reorder_queues(b);
        if (r != FE2_OK) return r;
    }
    {
        const fe2_status r = warm_shapes(b, o);
        if (r != FE2_OK) return r;
    }
    int launches = 0, timed = 0;
    if (o.launch == 1) {
        const fe2_status r = record_solve(b, o, st, false, &launches, &timed);
        if (r != FE2_OK) return r;
    } else {
        // one CUDA graph per option set: captured on the first solve with
        // these options, replayed by every later one
        if (!b->graph || !same_solve_opts(b->graph_opts, o)) {
            if (b->graph) CUDA_TRY(cudaGraphExecDestroy(b->graph));
            b->graph = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            const fe2_status r = record_solve(b, o, b->cap, true, &launches, &timed);
            cudaGraph_t g = nullptr;
            const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
            if (r != FE2_OK) {
                if (g) cudaGraphDestroy(g);
                return r;
            }
            if (e != cudaSuccess) return fail(FE2_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
            cudaGraphDestroy(g);
            if (ei != cudaSuccess) {
                b->graph = nullptr;
                return fail(FE2_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
            }
            b->graph_opts = o;
            b->graph_launches = launches;
            b->graph_timed = timed;
        }
        CUDA_TRY(cudaGraphLaunch(b->graph, st));
        launches = b->graph_launches;
        timed = b->graph_timed;
    }
    b->last_launches = launches;
    b->last_energy = o.kinetic_energy;
    b->last_timed = timed / 2;
    b->last_stream = st;
    b->solved = true;
    CUDA_TRY(cudaEventRecord(b->ev_done, st));
    return FE2_OK;
}

}  // namespace

extern "C" fe2_status fe2_batch_solve_dev(fe2_batch *b, const double *F_dev, const fe2_opts *opts,
                                          void *stream) {
    if (!b || !F_dev) return fail(FE2_EINVAL, "NULL batch or F");
    fe2_opts o;
    if (opts) o = *opts; else fe2_opts_default(&o);
    fe2_status s = check_opts(o);
    if (s != FE2_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = after_slots(b, st);
    if (s != FE2_OK) return s;
    CUDA_TRY(cudaMemcpyAsync(b->d_F.p, F_dev, sizeof(double) * 9 * b->n_rve,
                             cudaMemcpyDeviceToDevice, st));
    return launch_solve(b, o, st);
}

extern "C" fe2_status fe2_batch_solve(fe2_batch *b, const double *F, const fe2_opts *opts,
                                      void *stream) {
    if (!b || !F) return fail(FE2_EINVAL, "NULL batch or F");
    fe2_opts o;
    if (opts) o = *opts; else fe2_opts_default(&o);
    fe2_status s = check_opts(o);
    if (s != FE2_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Stage F in pinned memory so the caller's buffer is free on return; the
    // previous solve's upload from the staging buffer must have completed.
    CUDA_TRY(cudaEventSynchronize(b->ev_F));
    s = after_slots(b, st);
    if (s != FE2_OK) return s;
    std::memcpy(b->h_F, F, sizeof(double) * 9 * b->n_rve);
    CUDA_TRY(cudaMemcpyAsync(b->d_F.p, b->h_F, sizeof(double) * 9 * b->n_rve, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaEventRecord(b->ev_F, st));
    return launch_solve(b, o, st);
}

extern "C" fe2_status fe2_batch_stress(fe2_batch *b, double *sigma, int64_t *iters, double *rel_res,
                                       int32_t *status) {
    if (!b) return fail(FE2_EINVAL, "NULL batch");
    if (!b->solved) return fail(FE2_ESTATE, "no solve has been issued");
    CUDA_TRY(cudaStreamSynchronize(b->last_stream));
    {
        const fe2_status w = wait_slots(b);
        if (w != FE2_OK) return w;
    }
    const size_t P = b->n_rve;
    if (sigma) CUDA_TRY(cudaMemcpy(sigma, b->d_sigma.p, sizeof(double) * 9 * P, cudaMemcpyDeviceToHost));
    if (iters) CUDA_TRY(cudaMemcpy(iters, b->d_iters.p, sizeof(int64_t) * P, cudaMemcpyDeviceToHost));
    if (rel_res) CUDA_TRY(cudaMemcpy(rel_res, b->d_rel.p, sizeof(double) * P, cudaMemcpyDeviceToHost));
    if (status) CUDA_TRY(cudaMemcpy(status, b->d_status.p, sizeof(int32_t) * P, cudaMemcpyDeviceToHost));
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_diagnostics(fe2_batch *b, double *f_ref, double *kinetic_energy,
                                            int64_t *lead_iters) {
    if (!b) return fail(FE2_EINVAL, "NULL batch");
    if (!b->solved) return fail(FE2_ESTATE, "no solve has been issued");
    CUDA_TRY(cudaStreamSynchronize(b->last_stream));
    {
        const fe2_status w = wait_slots(b);
        if (w != FE2_OK) return w;
    }
    const size_t P = b->n_rve;
    if (f_ref) CUDA_TRY(cudaMemcpy(f_ref, b->d_fref.p, sizeof(double) * P, cudaMemcpyDeviceToHost));
    if (kinetic_energy) CUDA_TRY(cudaMemcpy(kinetic_energy, b->d_ke.p, sizeof(double) * P, cudaMemcpyDeviceToHost));
    if (lead_iters) CUDA_TRY(cudaMemcpy(lead_iters, b->d_lead.p, sizeof(int64_t) * P, cudaMemcpyDeviceToHost));
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_energy(fe2_batch *b, double *kinetic, double *internal_work,
                                        double *external_work, double *balance) {
    if (!b) return fail(FE2_EINVAL, "NULL batch");
    if (!b->solved) return fail(FE2_ESTATE, "no solve has been issued");
    if (b->last_energy != 2) return fail(FE2_ESTATE, "the last solve did not track the energy balance");
    CUDA_TRY(cudaStreamSynchronize(b->last_stream));
    {
        const fe2_status w = wait_slots(b);
        if (w != FE2_OK) return w;
    }
    const size_t P = b->n_rve;
    std::vector<double> k(P), wi(P), we(P);
    CUDA_TRY(cudaMemcpy(k.data(), b->d_ke.p, sizeof(double) * P, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(wi.data(), b->d_wint.p, sizeof(double) * P, cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(we.data(), b->d_wext.p, sizeof(double) * P, cudaMemcpyDeviceToHost));
    for (size_t p = 0; p < P; ++p) {
        if (kinetic) kinetic[p] = k[p];
        if (internal_work) internal_work[p] = wi[p];
        if (external_work) external_work[p] = we[p];
        if (balance) {
            const double scale = std::max(std::max(std::fabs(wi[p]), std::fabs(we[p])), k[p]);
            const double err = k[p] + wi[p] - we[p];
            balance[p] = scale > 0.0 ? err / scale : 0.0;
        }
    }
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_results_dev(fe2_batch *b, double *sigma_dev, int64_t *iters_dev,
                                            double *rel_res_dev, int32_t *status_dev, void *stream) {
    if (!b) return fail(FE2_EINVAL, "NULL batch");
    if (!b->solved) return fail(FE2_ESTATE, "no solve has been issued");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, b->ev_done, 0));
    {
        const fe2_status w = after_slots(b, st);
        if (w != FE2_OK) return w;
    }
    const size_t P = b->n_rve;
    if (sigma_dev) CUDA_TRY(cudaMemcpyAsync(sigma_dev, b->d_sigma.p, sizeof(double) * 9 * P, cudaMemcpyDeviceToDevice, st));
    if (iters_dev) CUDA_TRY(cudaMemcpyAsync(iters_dev, b->d_iters.p, sizeof(int64_t) * P, cudaMemcpyDeviceToDevice, st));
    if (rel_res_dev) CUDA_TRY(cudaMemcpyAsync(rel_res_dev, b->d_rel.p, sizeof(double) * P, cudaMemcpyDeviceToDevice, st));
    if (status_dev) CUDA_TRY(cudaMemcpyAsync(status_dev, b->d_status.p, sizeof(int32_t) * P, cudaMemcpyDeviceToDevice, st));
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_get_displacement(fe2_batch *b, double *u) {
    if (!b || !u) return fail(FE2_EINVAL, "NULL batch or u");
    if (b->solved) CUDA_TRY(cudaStreamSynchronize(b->last_stream));
    {
        const fe2_status w = wait_slots(b);
        if (w != FE2_OK) return w;
    }
    const int64_t N = b->n_nodes;
    std::vector<double> h(3 * N);
    CUDA_TRY(cudaMemcpy(h.data(), b->d_u.p, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < N; ++k) {
        const int64_t o = b->perm_to_orig[k];
        for (int r = 0; r < 3; ++r) u[3 * o + r] = h[r * N + k];
    }
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_set_displacement(fe2_batch *b, const double *u) {
    if (!b || !u) return fail(FE2_EINVAL, "NULL batch or u");
    const int64_t N = b->n_nodes;
    for (int64_t k = 0; k < 3 * N; ++k)
        if (!std::isfinite(u[k])) return fail(FE2_EINVAL, "non-finite displacement");
    if (b->solved) CUDA_TRY(cudaStreamSynchronize(b->last_stream));
    {
        const fe2_status w = wait_slots(b);
        if (w != FE2_OK) return w;
    }
    std::vector<double> h(3 * N);
    for (int64_t k = 0; k < N; ++k) {
        const int64_t o = b->perm_to_orig[k];
        for (int r = 0; r < 3; ++r) h[r * N + k] = u[3 * o + r];
    }
    CUDA_TRY(cudaMemcpy(b->d_u.p, h.data(), sizeof(double) * 3 * N, cudaMemcpyHostToDevice));
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_info(const fe2_batch *b, int32_t *n_rve, int64_t *n_nodes,
                                     int64_t *n_elems, int32_t *launches) {
    if (!b) return fail(FE2_EINVAL, "NULL batch");
    if (n_rve) *n_rve = b->n_rve;
    if (n_nodes) *n_nodes = b->n_nodes;
    if (n_elems) *n_elems = b->n_elems;
    if (launches) *launches = b->last_launches;
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_kernel_times(fe2_batch *b, float *ms, int32_t cap, int32_t *n) {
    if (!b || !n) return fail(FE2_EINVAL, "NULL batch or n");
    if (!b->solved) return fail(FE2_ESTATE, "no solve has been issued");
    *n = b->last_timed;
    for (int32_t k = 0; k < b->last_timed && k < cap; ++k) {
        CUDA_TRY(cudaEventSynchronize(b->tev[2 * k + 1]));
        CUDA_TRY(cudaEventElapsedTime(ms + k, b->tev[2 * k], b->tev[2 * k + 1]));
    }
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_parts(const fe2_batch *b, int32_t *parts) {
    if (!b || !parts) return fail(FE2_EINVAL, "NULL batch or parts");
    for (int32_t p = 0; p < b->n_rve; ++p) parts[p] = b->rve[p].n_parts;
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_destroy(fe2_batch *b) {
    if (!b) return FE2_OK;
    if (b->solved && b->last_stream) cudaStreamSynchronize(b->last_stream);
    cudaDeviceSynchronize();
    b->release();
    delete b;
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_solve_naive(fe2_batch *b, const double *F, const fe2_opts *opts,
                                            void *stream) {
    if (!b || !F) return fail(FE2_EINVAL, "NULL batch or F");
    fe2_opts o;
    if (opts) o = *opts; else fe2_opts_default(&o);
    fe2_status s = check_opts(o);
    if (s != FE2_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int64_t nmax = 0;
    for (auto &R : b->rve) nmax = std::max<int64_t>(nmax, R.n_nodes);
    if (!b->d_naive.p) CUDA_TRY(b->d_naive.alloc(6 * nmax + 16));
    CUDA_TRY(cudaStreamWaitEvent(st, b->ev_done, 0));
    s = after_slots(b, st);
    if (s != FE2_OK) return s;
    CUDA_TRY(cudaMemcpyAsync(b->d_F.p, F, sizeof(double) * 9 * b->n_rve, cudaMemcpyHostToDevice, st));
    NaiveScratch W;
    W.x = b->d_naive.p;
    W.g = b->d_naive.p + 3 * nmax;
    W.acc = b->d_naive.p + 6 * nmax;
    const DevMesh M = b->mesh();
    const DevState S = b->state();
    const DevResults R = b->results();
    std::vector<int64_t> iters(b->n_rve);
    std::vector<double> rel(b->n_rve);
    std::vector<int32_t> stat(b->n_rve);
    int launches = 0;
    for (int32_t p = 0; p < b->n_rve; ++p) {
        int stt = 0;
        const int e = naive_solve_rve(b->rve[p], M, S, R, b->d_F.p, W, o.tol, o.max_iter,
                                      o.dt_safety, o.init, p, st, &iters[p], &rel[p], &stt);
        if (e != 0) return fail(FE2_ECUDA, std::string("naive: ") + cudaGetErrorString((cudaError_t)e));
        stat[p] = stt;
        launches += 10 + 4 * (int)iters[p];
    }
    CUDA_TRY(cudaMemcpyAsync(b->d_iters.p, iters.data(), sizeof(int64_t) * b->n_rve, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(b->d_rel.p, rel.data(), sizeof(double) * b->n_rve, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(b->d_status.p, stat.data(), sizeof(int32_t) * b->n_rve, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    b->last_launches = launches;
    b->last_energy = 0;
    b->last_timed = 0;
    b->last_stream = st;
    b->solved = true;
    return FE2_OK;
}

// ---------------------------------------------------------------------------
// Serving: continuous micro-batching. A submission stages the deformation
// gradients of a set of RVEs, launches the solver for just those RVEs on a
// stream of its own (so in-flight submissions overlap on the device) and
// queues the copy of their results; poll hands back finished submissions.
// Every RVE keeps its state on the device between submissions, which is what
// FE2_INIT_WARM restarts from.
// ---------------------------------------------------------------------------
namespace {

__global__ void k_scatter_F(int n, const int32_t *ids, const double *Fs, double *F) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 9 * n) return;
    F[9 * (int64_t)ids[t / 9] + t % 9] = Fs[t];
}

__global__ void k_gather_results(int n, const int32_t *ids, const double *sigma, const double *rel,
                                 const int64_t *iters, const int32_t *status, double *out,
                                 int64_t *it_out, int32_t *st_out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t p = ids[t];
    for (int k = 0; k < 9; ++k) out[10 * (int64_t)t + k] = sigma[9 * p + k];
    out[10 * (int64_t)t + 9] = rel[p];
    it_out[t] = iters[p];
    st_out[t] = status[p];
}

double working_bytes(const fe2_batch *b, int32_t p) {
    // device state a solve keeps busy: mixed staging + per-node solver arrays
    return 200.0 * (double)b->rve[p].n_nodes;
}

}  // namespace

extern "C" fe2_status fe2_batch_submit(fe2_batch *b, int32_t n, const int32_t *rve_ids,
                                       const double *F, const fe2_opts *opts, int32_t *ticket) {
    if (!b || !rve_ids || !F || n < 1) return fail(FE2_EINVAL, "NULL argument or n < 1");
    if (n > b->n_rve) return fail(FE2_EINVAL, "more RVEs than the batch holds");
    fe2_opts o;
    if (opts) o = *opts; else fe2_opts_default(&o);
    fe2_status st = check_opts(o);
    if (st != FE2_OK) return st;
    for (int32_t k = 0; k < n; ++k) {
        if (rve_ids[k] < 0 || rve_ids[k] >= b->n_rve) return fail(FE2_EINVAL, "RVE id out of range");
        if (b->in_flight[rve_ids[k]]) return fail(FE2_EINVAL, "RVE " + std::to_string(rve_ids[k]) + " is already in flight");
    }
    int slot = -1;
    for (size_t k = 0; k < b->slots.size(); ++k)
        if (!b->slots[k].busy) { slot = (int)k; break; }
    if (slot < 0) return fail(FE2_EBUSY, "every serving slot is in flight");
    b->last_energy = 0;  // the submission rewrites part of the per-RVE results
    ServeSlot &sl = b->slots[slot];
    const bool fp64 = o.precision == FE2_PREC_FP64;
    auto &classes = fp64 ? b->classes_fp64 : b->classes_mixed;
    auto &class_of = fp64 ? b->class_of_fp64 : b->class_of_mixed;
    // staged ids, then the ids again grouped by class (largest first)
    std::vector<std::vector<int32_t>> per(classes.size());
    for (int32_t k = 0; k < n; ++k) {
        // mark duplicates within one submission as errors
        for (int32_t j = 0; j < k; ++j)
            if (rve_ids[j] == rve_ids[k]) return fail(FE2_EINVAL, "RVE id repeated in one submission");
        per[class_of[rve_ids[k]]].push_back(rve_ids[k]);
        sl.h_ids[k] = rve_ids[k];
    }
    int32_t off = n;
    std::vector<std::pair<int, int32_t>> starts;
    for (size_t c = 0; c < per.size(); ++c) {
        std::stable_sort(per[c].begin(), per[c].end(), [&](int32_t x, int32_t y) {
            return b->rve[x].n_free > b->rve[y].n_free;
        });
        starts.emplace_back((int)c, off);
        for (int32_t id : per[c]) sl.h_ids[off++] = id;
    }
    std::memcpy(sl.h_F, F, sizeof(double) * 9 * n);
    cudaStream_t s = sl.stream;
    // after the last batched solve, which writes every RVE's state
    CUDA_TRY(cudaStreamWaitEvent(s, b->ev_done, 0));
    CUDA_TRY(cudaMemcpyAsync(sl.d_ids, sl.h_ids, sizeof(int32_t) * 2 * n, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(sl.d_F, sl.h_F, sizeof(double) * 9 * n, cudaMemcpyHostToDevice, s));
    k_scatter_F<<<(9 * n + 255) / 256, 256, 0, s>>>(n, sl.d_ids, sl.d_F, b->d_F.p);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemsetAsync(sl.d_cnt, 0, sizeof(int32_t) * kCountersPerClass * classes.size(), s));
    {
        const fe2_status r = warm_shapes(b, o);
        if (r != FE2_OK) return r;
    }
    const SolveParams P = make_params(b, o);
    int launches = 0;
    for (auto &[c, q0] : starts) {
        if (per[c].empty()) continue;
        const fe2_status r = launch_class(b, o, classes[c], P, sl.d_ids + q0, (int)per[c].size(),
                                          sl.d_cnt + kCountersPerClass * c, s, nullptr, &launches);
        if (r != FE2_OK) return r;
    }
    k_gather_results<<<(n + 127) / 128, 128, 0, s>>>(n, sl.d_ids, b->d_sigma.p, b->d_rel.p, b->d_iters.p,
                                                     b->d_status.p, sl.d_out, sl.d_it, sl.d_st);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(sl.h_out, sl.d_out, sizeof(double) * 10 * n, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(sl.h_it, sl.d_it, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(sl.h_st, sl.d_st, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaEventRecord(sl.done, s));
    sl.n = n;
    sl.busy = true;
    sl.bytes = 0.0;
    for (int32_t k = 0; k < n; ++k) {
        b->in_flight[rve_ids[k]] = 1;
        sl.bytes += working_bytes(b, rve_ids[k]);
    }
    b->solved = true;
    b->last_stream = s;
    if (ticket) *ticket = slot;
    return FE2_OK;
}

extern "C" fe2_status fe2_batch_poll(fe2_batch *b, int32_t max, int32_t *ids, double *sigma,
                                     int64_t *iters, double *rel_res, int32_t *status, int32_t *n_out) {
    if (!b || !n_out) return fail(FE2_EINVAL, "NULL batch or n_out");
    *n_out = 0;
    for (auto &sl : b->slots) {
        if (!sl.busy) continue;
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return fail(FE2_ECUDA, std::string("serving slot: ") + cudaGetErrorString(q));
        if (*n_out + sl.n > max) break;  // no room: leave it for the next poll
        for (int k = 0; k < sl.n; ++k) {
            const int o = *n_out + k;
            if (ids) ids[o] = sl.h_ids[k];
            if (sigma) std::memcpy(sigma + 9 * (int64_t)o, sl.h_out + 10 * (int64_t)k, sizeof(double) * 9);
            if (rel_res) rel_res[o] = sl.h_out[10 * (int64_t)k + 9];
            if (iters) iters[o] = sl.h_it[k];
            if (status) status[o] = sl.h_st[k];
            b->in_flight[sl.h_ids[k]] = 0;
        }
        *n_out += sl.n;
        sl.busy = false;
        sl.n = 0;
    }
    return FE2_OK;
}

extern "C" fe2_status fe2_serve(fe2_batch *b, int32_t n_req, const int32_t *rve, const double *t_arrive,
                                const double *F, const fe2_opts *opts_first, const fe2_opts *opts_next,
                                int32_t max_batch, double max_inflight_bytes, double *t_done,
                                int64_t *iters, int32_t *status, double *sigma) {
    if (!b || n_req < 0 || (n_req > 0 && (!rve || !t_arrive || !F || !t_done)))
        return fail(FE2_EINVAL, "NULL argument");
    if (max_batch < 1) max_batch = b->n_rve;
    for (int32_t r = 0; r < n_req; ++r) {
        if (rve[r] < 0 || rve[r] >= b->n_rve) return fail(FE2_EINVAL, "request RVE id out of range");
        if (r > 0 && t_arrive[r] < t_arrive[r - 1]) return fail(FE2_EINVAL, "arrival times must not decrease");
    }
    for (auto &sl : b->slots)
        if (sl.busy) return fail(FE2_ESTATE, "serving slots are busy; poll them first");
    // per RVE: its requests in arrival order; a request becomes eligible once it
    // has arrived and the previous request of its RVE has completed
    std::vector<std::vector<int32_t>> chain(b->n_rve);
    for (int32_t r = 0; r < n_req; ++r) chain[rve[r]].push_back(r);
    std::vector<int32_t> next(b->n_rve, 0);           // index into chain of the next request
    std::vector<int32_t> running(b->n_rve, -1);       // request in flight per RVE
    std::vector<uint8_t> seen(b->n_rve, 0);           // RVE already solved once (warm start)
    std::vector<int32_t> ids(b->n_rve), done_ids(b->n_rve);
    std::vector<double> Fs(9 * (size_t)b->n_rve), sig(9 * (size_t)b->n_rve), rr(b->n_rve);
    std::vector<int64_t> its(b->n_rve);
    std::vector<int32_t> sts(b->n_rve);
    fe2_opts of, on;
    if (opts_first) of = *opts_first; else fe2_opts_default(&of);
    if (opts_next) on = *opts_next; else { on = of; on.init = FE2_INIT_WARM; }
    int32_t completed = 0;
    double inflight = 0.0;
    const auto t0 = std::chrono::steady_clock::now();
    auto now = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
    while (completed < n_req) {
        // completions
        int32_t got = 0;
        fe2_status st = fe2_batch_poll(b, b->n_rve, done_ids.data(), sig.data(), its.data(), rr.data(),
                                       sts.data(), &got);
        if (st != FE2_OK) return st;
        const double tn = now();
        for (int32_t k = 0; k < got; ++k) {
            const int32_t p = done_ids[k], r = running[p];
            t_done[r] = tn;
            if (iters) iters[r] = its[k];
            if (status) status[r] = sts[k];
            if (sigma) std::memcpy(sigma + 9 * (int64_t)r, sig.data() + 9 * (size_t)k, sizeof(double) * 9);
            running[p] = -1;
            inflight -= working_bytes(b, p);
            ++completed;
        }
        // admission: arrived, eligible, within slots and the working-set budget
        for (int pass = 0; pass < 2; ++pass) {  // first solves, then warm restarts
            const bool warm = pass == 1;
            int32_t n = 0;
            for (int32_t p = 0; p < b->n_rve && n < max_batch; ++p) {
                if (running[p] >= 0 || next[p] >= (int32_t)chain[p].size()) continue;
                if ((seen[p] != 0) != warm) continue;
                const int32_t r = chain[p][next[p]];
                if (t_arrive[r] > tn) continue;
                const double wb = working_bytes(b, p);
                if (max_inflight_bytes > 0.0 && inflight + wb > max_inflight_bytes && inflight > 0.0) continue;
                ids[n] = p;
                std::memcpy(Fs.data() + 9 * (size_t)n, F + 9 * (int64_t)r, sizeof(double) * 9);
                inflight += wb;
                ++n;
            }
            if (n == 0) continue;
            int32_t ticket = -1;
            st = fe2_batch_submit(b, n, ids.data(), Fs.data(), warm ? &on : &of, &ticket);
            if (st == FE2_EBUSY) {  // no free slot: undo and retry after the next poll
                for (int32_t k = 0; k < n; ++k) inflight -= working_bytes(b, ids[k]);
                break;
            }
            if (st != FE2_OK) return st;
            for (int32_t k = 0; k < n; ++k) {
                const int32_t p = ids[k];
                running[p] = chain[p][next[p]];
                ++next[p];
                seen[p] = 1;
            }
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    return FE2_OK;
}

// ---------------------------------------------------------------------------
// Launch tuning and the autotuner (Section III: the best number of threads
// per team depends on the sub-problem size). A configuration per size bucket:
// cluster size and FP32-kernel CTA size, chosen by timing bounded solves.
// ---------------------------------------------------------------------------
namespace {

fe2_status check_tuning(const fe2_tuning &t) {
    for (int k = 0; k < 32; ++k) {
        const int c = t.parts[k];
        if (c < 0 || c > kMaxParts || (c & (c - 1)) != 0) return fail(FE2_EINVAL, "tuning: parts must be 0 or a power of two <= 16");
        for (int v : {t.block_fp32[k], t.block_lead[k]})
            if (v != 0 && (v < 64 || v > 512 || v % 32)) return fail(FE2_EINVAL, "tuning: CTA sizes must be 0 or multiples of 32 in [64, 512]");
    }
    return FE2_OK;
}

// The value of "key": <number> inside text[lo, hi), or NAN.
double json_num(const std::string &text, size_t lo, size_t hi, const char *key) {
    const std::string k = std::string("\"") + key + "\"";
    const size_t at = text.find(k, lo);
    if (at == std::string::npos || at >= hi) return NAN;
    size_t c = text.find(':', at + k.size());
    if (c == std::string::npos || c >= hi) return NAN;
    return std::strtod(text.c_str() + c + 1, nullptr);
}
std::string json_str(const std::string &text, const char *key) {
    const std::string k = std::string("\"") + key + "\"";
    const size_t at = text.find(k);
    if (at == std::string::npos) return "";
    const size_t q0 = text.find('"', text.find(':', at + k.size()));
    if (q0 == std::string::npos) return "";
    const size_t q1 = text.find('"', q0 + 1);
    return q1 == std::string::npos ? "" : text.substr(q0 + 1, q1 - q0 - 1);
}

struct DeviceId {
    std::string name;
    int sms = 0;
};
fe2_status device_id(DeviceId &d) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    d.name = prop.name;
    d.sms = prop.multiProcessorCount;
    return FE2_OK;
}

}  // namespace

extern "C" fe2_status fe2_tuning_set(const fe2_tuning *t) {
    if (!t) {
        g_tuning = fe2_tuning{};
        return FE2_OK;
    }
    const fe2_status s = check_tuning(*t);
    if (s != FE2_OK) return s;
    g_tuning = *t;
    return FE2_OK;
}

extern "C" fe2_status fe2_tuning_get(fe2_tuning *t) {
    if (!t) return fail(FE2_EINVAL, "NULL tuning");
    *t = g_tuning;
    return FE2_OK;
}

extern "C" fe2_status fe2_tuning_load(const char *path) {
    if (!path) return fail(FE2_EINVAL, "NULL path");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(FE2_EINVAL, std::string("cannot read ") + path);
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    DeviceId d;
    const fe2_status ds = device_id(d);
    if (ds != FE2_OK) return ds;
    if (json_str(text, "gpu") != d.name || (int)json_num(text, 0, text.size(), "sm_count") != d.sms)
        return fail(FE2_EINVAL, std::string("tuning file ") + path + " was measured on another GPU");
    if (json_str(text, "precision") != "mixed") return fail(FE2_EINVAL, "tuning file is not for the mixed solver");
    fe2_tuning t = {};
    const size_t arr = text.find("\"buckets\"");
    if (arr == std::string::npos) return fail(FE2_EINVAL, "tuning file has no buckets");
    // every object after the key is one bucket (objects hold no nested objects)
    size_t pos = arr;
    while (true) {
        const size_t o0 = text.find('{', pos);
        if (o0 == std::string::npos) break;
        const size_t o1 = text.find('}', o0);
        if (o1 == std::string::npos) return fail(FE2_EINVAL, "tuning file is malformed");
        const double b = json_num(text, o0, o1, "bucket"), c = json_num(text, o0, o1, "parts"),
                     k = json_num(text, o0, o1, "block_fp32");
        if (!(b >= 0 && b < 32) || std::isnan(c) || std::isnan(k)) return fail(FE2_EINVAL, "tuning file is malformed");
        t.parts[(int)b] = (int32_t)c;
        t.block_fp32[(int)b] = (int32_t)k;
        pos = o1 + 1;
    }
    return fe2_tuning_set(&t);
}

extern "C" fe2_status fe2_autotune(int32_t n_rve, const int64_t *node_off, const double *X,
                                   const int64_t *elem_off, const int32_t *conn, const double *EA,
                                   const uint8_t *fixed, const double *damping, const double *F,
                                   int64_t trial_iters, const char *json_path, fe2_tuning *out) {
    {
        const fe2_status v = validate_batch(n_rve, node_off, X, elem_off, conn, EA, fixed, nullptr, damping);
        if (v != FE2_OK) return v;
    }
    if (!F) return fail(FE2_EINVAL, "NULL F");
    if (trial_iters < 8) return fail(FE2_EINVAL, "trial_iters must be >= 8");
    DeviceId dev;
    {
        const fe2_status ds = device_id(dev);
        if (ds != FE2_OK) return ds;
    }
    int devi = 0;
    CUDA_TRY(cudaGetDevice(&devi));
    size_t optin = 0;
    {
        cudaDeviceProp prop;
        CUDA_TRY(cudaGetDeviceProperties(&prop, devi));
        optin = prop.sharedMemPerBlockOptin;
    }
    const int target = std::max(64, env_int("FE2_NODES_PER_CTA", 1024));
    const fe2_tuning saved = g_tuning;
    fe2_tuning best = saved;
    std::vector<std::vector<int32_t>> by_bucket(32);
    for (int32_t p = 0; p < n_rve; ++p) by_bucket[node_bucket((int)(node_off[p + 1] - node_off[p]))].push_back(p);
    cudaStream_t st = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    CUDA_TRY(cudaEventCreate(&t0));
    CUDA_TRY(cudaEventCreate(&t1));
    std::string report;
    fe2_status rc = FE2_OK;
    for (int bk = 0; bk < 32 && rc == FE2_OK; ++bk) {
        const auto &S = by_bucket[bk];
        if (S.empty()) continue;
        int cmin = 1;
        for (int32_t p : S) cmin = std::max(cmin, min_parts((int)(node_off[p + 1] - node_off[p]), target, optin - 16384));
        double best_rate = -1.0;
        int best_c = 0, best_blk = 0;
        std::string tried;
        for (int C = cmin; C <= kMaxParts && rc == FE2_OK; C *= 2) {
            // the bucket's samples, replicated until they fill every SM once
            const int want = std::max<int>((int)S.size(), (dev.sms + C - 1) / C);
            std::vector<int64_t> no(1, 0), eo(1, 0);
            std::vector<double> x, ea, damp, f;
            std::vector<int32_t> cn;
            std::vector<uint8_t> fx;
            for (int k = 0; k < want; ++k) {
                const int32_t p = S[k % S.size()];
                const int64_t n0 = node_off[p], n1 = node_off[p + 1], e0 = elem_off[p], e1 = elem_off[p + 1];
                x.insert(x.end(), X + 3 * n0, X + 3 * n1);
                fx.insert(fx.end(), fixed + n0, fixed + n1);
                cn.insert(cn.end(), conn + 2 * e0, conn + 2 * e1);
                ea.insert(ea.end(), EA + e0, EA + e1);
                damp.push_back(damping ? damping[p] : 0.002 * std::cbrt(512.0 / (double)(n1 - n0)));
                f.insert(f.end(), F + 9 * (int64_t)p, F + 9 * (int64_t)p + 9);
                no.push_back(no.back() + (n1 - n0));
                eo.push_back(eo.back() + (e1 - e0));
            }
            g_tuning = saved;
            g_tuning.parts[bk] = C;
            g_tuning.block_fp32[bk] = 0;
            fe2_batch *tb = nullptr;
            fe2_status cs = fe2_batch_create(want, no.data(), x.data(), eo.data(), cn.data(), ea.data(), fx.data(),
                                             nullptr, damp.data(), st, &tb);
            if (cs != FE2_OK) {
                if (cs == FE2_ENOMEM) break;
                rc = cs;
                break;
            }
            bool forced_ok = true;
            for (int32_t p = 0; p < want; ++p) forced_ok &= tb->rve[p].n_parts == C;
            for (int blk : {256, 384, 512}) {
                if (!forced_ok) break;
                for (auto &c : tb->classes_mixed) c.block_fp32 = blk;
                fe2_opts o;
                fe2_opts_default(&o);
                o.tol = 0.0;
                o.launch = 1;
                o.max_iter = 16;  // warm-up: attributes, occupancy
                o.lead_iters = 4;
                fe2_status ss = fe2_batch_solve(tb, f.data(), &o, st);
                if (ss == FE2_OK) ss = fe2_batch_stress(tb, nullptr, nullptr, nullptr, nullptr);
                if (ss != FE2_OK) {
                    if (ss == FE2_EINVAL) break;  // does not fit this cluster size
                    rc = ss;
                    break;
                }
                o.max_iter = trial_iters;
                o.lead_iters = trial_iters / 4;
                CUDA_TRY(cudaEventRecord(t0, st));
                ss = fe2_batch_solve(tb, f.data(), &o, st);
                if (ss != FE2_OK) { rc = ss; break; }
                CUDA_TRY(cudaEventRecord(t1, st));
                CUDA_TRY(cudaEventSynchronize(t1));
                float ms = 0.f;
                CUDA_TRY(cudaEventElapsedTime(&ms, t0, t1));
                std::vector<int64_t> it(want);
                ss = fe2_batch_stress(tb, nullptr, it.data(), nullptr, nullptr);
                if (ss != FE2_OK) { rc = ss; break; }
                double work = 0.0;
                for (int32_t p = 0; p < want; ++p) work += (double)(no[p + 1] - no[p]) * (double)it[p];
                const double used = std::min<double>(dev.sms, (double)want * C);
                const double rate = work / (ms * 1e-3) / used;
                char line[96];
                std::snprintf(line, sizeof line, "%s[%d, %d, %.6g]", tried.empty() ? "" : ", ", C, blk, rate);
                tried += line;
                if (rate > best_rate) { best_rate = rate; best_c = C; best_blk = blk; }
            }
            fe2_batch_destroy(tb);
        }
        if (rc != FE2_OK) break;
        if (best_c > 0) {
            best.parts[bk] = best_c;
            best.block_fp32[bk] = best_blk;
            char line[256];
            std::snprintf(line, sizeof line,
                          "%s  {\"bucket\": %d, \"nodes_lo\": %lld, \"nodes_hi\": %lld, \"samples\": %zu, "
                          "\"parts\": %d, \"block_fp32\": %d, \"node_iters_per_s_per_sm\": %.6g, \"tried\": [",
                          report.empty() ? "" : ",\n", bk, (long long)1 << bk, ((long long)2 << bk) - 1, S.size(),
                          best_c, best_blk, best_rate);
            report += line;
            report += tried + "]}";
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaStreamDestroy(st);
    g_tuning = saved;
    if (rc != FE2_OK) return rc;
    g_tuning = best;
    if (out) *out = best;
    if (json_path) {
        FILE *f = std::fopen(json_path, "wb");
        if (!f) return fail(FE2_EINVAL, std::string("cannot write ") + json_path);
        std::fprintf(f,
                     "{\"gpu\": \"%s\", \"sm_count\": %d, \"precision\": \"mixed\", \"trial_iters\": %lld,\n"
                     " \"objective\": \"node-iterations per second per SM over bounded solves\",\n"
                     " \"tried_columns\": [\"parts\", \"block_fp32\", \"node_iters_per_s_per_sm\"],\n"
                     " \"buckets\": [\n%s\n]}\n",
                     dev.name.c_str(), dev.sms, (long long)trial_iters, report.c_str());
        std::fclose(f);
    }
    return FE2_OK;
}

// ---------------------------------------------------------------------------
// Sharding over GPUs (Section I: the microscale problems are independent).
// Longest-processing-time-first assignment of RVEs to ranks by estimated cost;
// the only exchange is gathering the 9-double stresses afterwards.
// ---------------------------------------------------------------------------
extern "C" fe2_status fe2_shard_plan(int32_t n_rve, const int64_t *node_off, const int64_t *iters,
                                     int32_t n_ranks, int32_t *rank_of, double *rank_cost) {
    if (n_rve < 0 || !node_off || n_ranks < 1 || (n_rve > 0 && !rank_of))
        return fail(FE2_EINVAL, "NULL argument, n_rve < 0 or n_ranks < 1");
    std::vector<double> cost(n_rve);
    for (int32_t p = 0; p < n_rve; ++p) {
        const double n = (double)(node_off[p + 1] - node_off[p]);
        if (!(n > 0)) return fail(FE2_EINVAL, "RVE " + std::to_string(p) + " has no nodes");
        // measured iterations when given, else the growth of the iteration
        // count with size seen on kNN networks (about n^0.5), so cost ~ n^1.5
        cost[p] = iters && iters[p] > 0 ? n * (double)iters[p] : n * std::sqrt(n);
    }
    std::vector<int32_t> order(n_rve);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    std::vector<double> load(n_ranks, 0.0);
    for (int32_t p : order) {
        int32_t r = 0;
        for (int32_t k = 1; k < n_ranks; ++k)
            if (load[k] < load[r]) r = k;
        rank_of[p] = r;
        load[r] += cost[p];
    }
    if (rank_cost) std::copy(load.begin(), load.end(), rank_cost);
    return FE2_OK;
}
