// Internal device/host data layout of a batch (not part of the C ABI).
//
// Packed, CRS-like storage of many RVEs (the paper's PackedView: a row-offset
// vector plus value vectors holding every sub-problem of a rank contiguously,
// Section III), re-laid out for the GPU:
//   * nodes of RVE p occupy [node0, node0 + n_nodes) of every node array, free
//     nodes first (the paper's free/fixed reordering, Section III), free nodes
//     sorted by degree so that a warp's gathers have equal trip counts;
//   * each node has a CSR row of its incident elements (node-centric, so the
//     force gather needs no atomics), ordered by the neighbour's ORIGINAL id:
//     this is the order in which a serial element scatter over lexicographic
//     (a < b) elements touches the node, which keeps FP64 sums bit-identical;
//   * structure-of-arrays per component for coalesced access.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

namespace fe2 {

struct RveDesc {
    int64_t node0;    // first node (permuted, global index)
    int64_t rp0;      // first row pointer: rowptr[rp0 .. rp0 + n_nodes]
    int64_t csr0;     // rowptr values are relative to this CSR entry
    int64_t elem0;    // first element of the stress list
    int32_t n_nodes;
    int32_t n_free;
    int32_t n_elems;
    int32_t max_deg;
    double dtc;       // critical time step (safety factor not applied)
    double c;         // damping coefficient
    double V0;        // reference volume
    double pad;
};

// Read-only, create-time arrays.
struct DevMesh {
    const RveDesc *rve;
    const double *X0, *X1, *X2;   // reference coordinates (permuted)
    const double *mass;           // lumped nodal mass
    const float *inv_mass_f;      // 1/m in FP32
    const int32_t *rowptr;        // per RVE n_nodes + 1 entries
    const int32_t *col;           // neighbour (local permuted id)
    const double *EA;             // per CSR entry
    const double *L;              // per CSR entry
    const float2 *EAf_invLf;      // per CSR entry: (EA, 1/L) in FP32
    const int32_t *el_a, *el_b;   // stress elements (local permuted ids)
    const double *el_EA, *el_L;
};

// Mutable solver state (device).
struct DevState {
    double *u0, *u1, *u2;         // displacement (output of every mode)
    double *v0, *v1, *v2;         // FP64 velocity
    double *a0, *a1, *a2;         // FP64 acceleration
    float *fv, *fa, *fg;          // MIXED: FP32 velocity, acceleration, g_ref (3*N each, SoA)
    double *xg;                   // 3*N global position scratch (RVEs too big for SMEM)
    float4 *pg;                   // 2*N float4 scratch (mixed positions, big RVEs)
};

struct DevResults {
    double *sigma;    // 9 per RVE
    int64_t *iters;
    double *rel_res;
    int32_t *status;
    double *f_ref;
    double *ke;
};

struct SolveParams {
    const double *F;      // 9 per RVE (device)
    double tol;
    int64_t max_iter;
    double alpha;
    int init;
    int want_ke;
    int64_t lead_iters;   // < 0: default rule
    int rebase_every;
    const int32_t *queue; // RVE ids in scheduling order
    int32_t queue_len;
    int32_t *counter;     // work-queue head (zeroed before the launch)
    int smem_positions;   // 1: positions staged in shared memory
};

enum { RVE_OK = 0, RVE_MAXITER = 1, RVE_NAN = 2, RVE_PENDING = 3 };

// Kernel launchers (defined in the .cu files).
int launch_setup(int32_t n_rve, int64_t n_el, int64_t n_csr, RveDesc *rve,
                 const int64_t *ga, const int64_t *gb, const double *X0, const double *X1,
                 const double *X2, const int64_t *elem_of, const double *EA_csr,
                 const double *el_EA, const int32_t *rowptr, double *el_L, double *L_csr,
                 float2 *eaf, double *mass, float *inv_mass_f, void *stream);
int launch_dr_fp64(const DevMesh &m, const DevState &s, const DevResults &r,
                   const SolveParams &p, int grid, int block, size_t smem, void *stream);
int launch_dr_mixed(const DevMesh &m, const DevState &s, const DevResults &r,
                    const SolveParams &p, int grid, int block, size_t smem, void *stream);
// Naive comparator: scratch sized for the largest RVE, and one RVE's solve.
struct NaiveScratch {
    double *x, *g, *acc;  // 3*n_max, 3*n_max, 16
};
int naive_solve_rve(const RveDesc &R, const DevMesh &M, const DevState &S, const DevResults &O,
                    const double *F_dev, const NaiveScratch &W, double tol, int64_t max_iter,
                    double alpha, int init, int p, cudaStream_t st, int64_t *iters_out,
                    double *rel_out, int *status_out);
// Resident CTAs per SM for a launch shape.
int occupancy_dr_fp64(int smem_positions, int block, size_t smem);
int occupancy_dr_mixed(int smem_positions, int block, size_t smem);

}  // namespace fe2
