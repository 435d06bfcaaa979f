// Internal device/host data layout of a batch (not part of the C ABI).
//
// Packed, CRS-like storage of many RVEs (the paper's PackedView: a row-offset
// vector plus value vectors holding every sub-problem of a rank contiguously,
// Section III), re-laid out for the GPU:
//   * nodes of RVE p occupy [node0, node0 + n_nodes) of every node array, free
//     nodes first (the paper's free/fixed reordering, Section III);
//   * an RVE is split spatially (recursive coordinate bisection) into
//     n_parts parts, one per CTA of the thread-block cluster that solves it in
//     mixed precision. Free nodes are ordered part by part (by degree within a
//     part), then fixed nodes part by part, so part r owns the free range
//     [part_f[r], part_f[r+1]) and the fixed range n_free + [part_g[r], part_g[r+1]);
//   * each node has a CSR row of its incident elements (node-centric, so the
//     force gather needs no atomics), ordered by the neighbour's ORIGINAL id:
//     the order in which a serial element scatter over lexicographic (a < b)
//     elements touches the node, which keeps FP64 sums bit-identical. `col`
//     holds the neighbour's RVE-local index, `col_part` the same neighbour as
//     (owning part << 16 | index inside that part's shared-memory arrays);
//   * structure-of-arrays per component for coalesced access.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fe2 {

constexpr int kMaxParts = 16;  // largest (non-portable) thread-block cluster

struct RveDesc {
    int64_t node0;    // first node (permuted, global index)
    int64_t rp0;      // first row pointer: rowptr[rp0 .. rp0 + n_nodes]
    int64_t csr0;     // rowptr values are relative to this CSR entry
    int64_t elem0;    // first element of the stress list
    int32_t n_nodes;
    int32_t n_free;
    int32_t n_elems;
    int32_t n_parts;  // cluster size of the mixed solver for this RVE
    double dtc;       // critical time step (safety factor not applied)
    double c;         // damping coefficient
    double V0;        // reference volume
    int32_t part_max;       // largest part (nodes), sizes the shared memory
    int32_t part_free_max;  // most free nodes in one part
    int32_t part_elem_max;  // FP32 kernel: most table elements of one part
    int32_t part_slot_max;  // FP32 kernel: most row slots (ELL, 32-node slabs) of one part
    int64_t slot0;          // FP64 cluster kernel: first element slot of this RVE
    int32_t part_fslot_max; // FP64 cluster kernel: most element slots of one part
    int32_t pad_;
};

// Read-only, create-time arrays.
struct DevMesh {
    const RveDesc *rve;
    const double *X0, *X1, *X2;   // reference coordinates (permuted)
    const float *Xh, *Xl;         // reference coordinates as double-float, [3][N]
    const double *mass;           // lumped nodal mass
    const float *imh, *iml;       // 1/m as double-float
    const int32_t *rowptr;        // per RVE n_nodes + 1 entries
    const int32_t *col;           // neighbour (RVE-local permuted id)
    const int32_t *col_part;      // neighbour as (part << 16 | index in part)
    const int32_t *part_off;      // per RVE 2*(kMaxParts+1): part_f[], part_g[]
    const double *EA;             // per CSR entry
    const double *L;              // per CSR entry
    const float2 *eaf;            // per CSR entry: (EA, 1/L) double-float high parts
    const float2 *eaf_lo;         // per CSR entry: low parts
    const float4 *dh, *dl;        // per CSR entry: (X_j - X_i, L) as double-float hi / lo
    const int32_t *el_a, *el_b;   // stress elements (RVE-local permuted ids)
    const double *el_EA, *el_L;
    const int32_t *csr_el;        // per CSR entry: RVE-local element << 1, | 1 when
                                  // the row's node is the element's second node
                                  // (caller orientation)
    const int4 *fp_slot;          // FP64 cluster kernel, per element slot: (element,
                                  // first end, second end, 0), ends as (part << 16 | index)
    const int32_t *fp_csr_slot;   // per CSR entry of a free node: part-relative slot << 1
                                  // | 1 when the node is the element's second end
    const int32_t *fp_part_slot;  // per RVE kMaxParts+1 part slot offsets (from slot0)
};

// Mutable solver state (device).
struct DevState {
    double *u0, *u1, *u2;         // displacement (output of every mode)
    double *v0, *v1, *v2;         // FP64 velocity
    double *a0, *a1, *a2;         // FP64 acceleration
    float *uh, *ul;               // MIXED: displacement, double-float [3][N]
    float *vh, *vl;               // MIXED: velocity (lead: double-float; FP32 phase: vh)
    float *ah, *al;               // MIXED: acceleration (same convention)
    float *fg;                    // MIXED: reference force g_ref, FP32 [3][N]
    double *xg;                   // [3][N] FP64 positions scratch
    double *tf;                   // FP64: per element, its force on the first node (3)
    float4 *sv;                   // MIXED FP32 kernel without element table: per node
    float2 *sa;                   //   (v, a.x) and (a.y, a.z)
    double *gp, *fdp;             // FP64 energy check: previous internal and damping
                                  // force per free DOF [3][N]
    double *ualt;                 // FP64 cluster kernel: displacement of odd evaluations,
                                  // per RVE [3][n] at 3 node0
    double *fpt;                  // FP64 cluster kernel: element forces [3][part slots]
                                  // when the table does not fit in shared memory
};

struct DevResults {
    double *sigma;    // 9 per RVE
    int64_t *iters;
    double *rel_res;
    int32_t *status;
    double *f_ref;
    double *ke;
    int64_t *lead;    // MIXED: iterations run in the double-float lead
    double *wint;     // FP64 energy check: stored internal work since the start
    double *wext;     //   and work of the damping forces
};

struct SolveParams {
    const double *F;      // 9 per RVE (device)
    double tol;
    int64_t max_iter;
    double alpha;
    int init;
    int want_ke;          // 1: kinetic energy; 2 (FP64): also the work terms of the
                          // energy balance
    int64_t lead_iters;   // < 0: lead until the relative residual <= lead_tol
    double lead_tol;
    int rebase_every;
    const int32_t *queue; // RVE ids in scheduling order
    int32_t queue_len;
    int32_t *counter;     // work-queue heads (zeroed before the launch; mixed uses three)
    int smem_positions;   // FP64 kernel: 1 = positions staged in shared memory
    int64_t stall_window; // MIXED: FP32 evaluations without the squared residual
                          // falling to a quarter before the RVE is handed back
                          // to double-float; 0 = never
    int resume;           // MIXED lead kernel: 1 = resume launch (stalled RVEs only)
};

// RVE_STALLED (internal): the FP32 phase stopped making progress and the RVE
// waits for the double-float resume launch, which replaces the status.
enum { RVE_OK = 0, RVE_MAXITER = 1, RVE_NAN = 2, RVE_PENDING = 3, RVE_STALLED = 5 };
// Work-queue heads per launch class: lead, FP32 phase, double-float resume.
constexpr int kCountersPerClass = 3;

// Kernel launchers (defined in the .cu files).
int launch_setup(int32_t n_rve, int64_t n_el, int64_t n_csr, RveDesc *rve,
                 const int64_t *ga, const int64_t *gb, const double *X0, const double *X1,
                 const double *X2, const int64_t *elem_of, const double *EA_csr,
                 const double *el_EA, const int32_t *rowptr, double *el_L, double *L_csr,
                 float2 *eaf, float2 *eaf_lo, double *mass, float *imh, float *iml,
                 float *Xh, float *Xl, const int32_t *col, float4 *dh, float4 *dl,
                 void *stream);
int launch_dr_fp64(const DevMesh &m, const DevState &s, const DevResults &r,
                   const SolveParams &p, int grid, int block, size_t smem, void *stream);
// Mixed solver: one thread-block cluster of `parts` CTAs per RVE; two
// persistent launches per class, the double-float lead (lead = 1) and then
// the FP32 phase (lead = 0).
int launch_dr_mixed(const DevMesh &m, const DevState &s, const DevResults &r,
                    const SolveParams &p, int lead, int clusters, int parts, int block,
                    size_t smem, int part_cap, int free_cap, int elem_cap, int slot_cap,
                    void *stream);
// Dynamic shared memory of the FP32 kernel for a class: the staged node state,
// plus each part's element table and rows when they fit within `limit` bytes.
size_t mixed_fp32_smem(int part_cap, int free_cap, int elem_cap, int slot_cap, size_t limit);
// Dynamic shared memory of the lead kernel for a class: one double-float
// displacement per node, or two plus the element table when they fit.
size_t mixed_lead_smem(int part_cap, int free_cap, int elem_cap, int slot_cap, size_t limit);
// Whether a launch with `smem` bytes uses the shared-memory element table.
bool mixed_staged(int lead, size_t smem, int part_cap);
// FP64 cluster kernel (dr_fp64_cluster.cu): dynamic shared memory (two
// position buffers, and the element table when tsm), launch, occupancy.
// ssm: the own free nodes' state (displacement, velocity, acceleration, mass)
// in shared memory as well.
size_t fp64_cluster_smem(int part_cap, int free_cap, int slot_cap, bool tsm, bool ssm);
int launch_dr_fp64_cluster(const DevMesh &m, const DevState &s, const DevResults &r, const SolveParams &p,
                           int clusters, int parts, int block, int part_cap, int free_cap, int slot_cap,
                           bool tsm, bool ssm, void *stream);
int occupancy_dr_fp64_cluster(int parts, int block, int part_cap, int free_cap, int slot_cap, bool tsm,
                              bool ssm);
// Shared memory per node of a kernel without its element table.
size_t mixed_plain_node_bytes(int lead);
// Resident CTAs per SM (FP64) / co-resident clusters (mixed) for a launch shape.
int occupancy_dr_fp64(int smem_positions, int block, size_t smem);
int occupancy_dr_mixed(int lead, int parts, int block, size_t smem, int part_cap);

// Naive comparator: scratch sized for the largest RVE, and one RVE's solve.
struct NaiveScratch {
    double *x, *g, *acc;  // 3*n_max, 3*n_max, 16
};
int naive_solve_rve(const RveDesc &R, const DevMesh &M, const DevState &S, const DevResults &O,
                    const double *F_dev, const NaiveScratch &W, double tol, int64_t max_iter,
                    double alpha, int init, int p, cudaStream_t st, int64_t *iters_out,
                    double *rel_out, int *status_out);

}  // namespace fe2
