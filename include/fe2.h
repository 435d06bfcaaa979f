/*
 * fe2.h - batched damped dynamic relaxation of many small fiber-network RVEs
 * on one GB300 GPU (sm_103a).
 *
 * Method: Merson & Shephard, "Using Hierarchical Parallelism to Accelerate the
 * Solution of Many Small Partial Differential Equations". In the FE2 scheme
 * every macroscale material point solves an independent microscale problem
 * (Section I); here that problem is a truss (fiber) network relaxed to static
 * equilibrium by damped explicit central-difference dynamics until the force
 * residual converges (Algorithm 1, Section III). Many such problems are packed
 * CRS-style, row offsets plus values, into one batch (the PackedView idea,
 * Section III) and solved together on the device.
 *
 * Conventions shared by every call:
 *   - Every call returns an fe2_status and never aborts or exits.
 *     fe2_last_error() gives a message for the last failing call of the
 *     calling thread.
 *   - Input arrays are caller-owned HOST memory unless a name ends in _dev.
 *     They are copied before the call returns (or, for the asynchronous _dev
 *     calls, read on the stream) and may be freed afterwards.
 *   - Node ids and element connectivity are exactly the caller's. Internal
 *     reorderings never show in any input or output.
 *   - 3x3 tensors (F, sigma) are row-major, 9 doubles per RVE.
 *   - A batch owns all of its device memory until fe2_batch_destroy(). The
 *     library allocates only in create and destroy; solve allocates nothing
 *     (the naive comparator, fe2_batch_solve_naive, allocates its scratch on
 *     first use).
 *   - Calls on one batch must not run concurrently from several host threads.
 *   - Serving submissions (fe2_batch_submit) and batched calls on the same
 *     batch are ordered: a submission starts after the last batched solve,
 *     a batched solve starts after every submission still in flight, and
 *     the host readbacks wait for both.
 */
#ifndef FE2_H
#define FE2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fe2_batch fe2_batch; /* opaque */

typedef enum {
    FE2_OK = 0,
    FE2_EINVAL = 1,   /* invalid argument or input data; nothing changed */
    FE2_ENOMEM = 2,   /* device or host allocation failed */
    FE2_ECUDA = 3,    /* a CUDA runtime call failed; see fe2_last_error() */
    FE2_ESTATE = 4,   /* call out of order (e.g. results before any solve) */
    FE2_ETIMEOUT = 5, /* a bounded device wait gave up (serving epochs) */
    FE2_ENODEV = 6,   /* no usable sm_103 device */
    FE2_EBUSY = 7     /* every serving slot is in flight; poll and retry */
} fe2_status;

/* Per-RVE outcome of a solve. */
typedef enum {
    FE2_RVE_OK = 0,      /* residual <= tol * f_ref */
    FE2_RVE_MAXITER = 1, /* max_iter iterations without converging */
    FE2_RVE_NAN = 2,     /* the residual became NaN or infinite */
    FE2_RVE_PENDING = 3  /* not solved yet (code 5 is internal: an RVE waiting
                            for the double-float resume; never returned) */
} fe2_rve_status;

typedef enum {
    /* IEEE FP64 in the order of the reference algorithm: the same operations
     * in the same order as a serial element-scatter implementation in the
     * caller's node order, no fused multiply-add, correctly rounded sqrt and
     * divide. The trajectory is bit for bit that of such an implementation;
     * only the residual and stress sums are reassociated. An RVE of one
     * spatial part runs on one CTA; an RVE of several parts on a
     * thread-block cluster, one part per CTA, with the same operations (set
     * FE2_FP64_CLUSTER=0 in the environment before fe2_batch_create to keep
     * every RVE on one CTA). Any RVE size. */
    FE2_PREC_FP64 = 0,
    /* All iteration arithmetic on the FP32 pipes, one thread-block cluster
     * of 1-16 CTAs per RVE: a double-float (FP32 pair) lead phase until the
     * relative residual drops below lead_tol (the transient in which the
     * network picks its equilibrium), then FP32 increments of the element
     * forces about a double-float reference state refreshed every
     * rebase_every iterations. The residual is totalled in double-float and
     * compared with (tol f_ref)^2 formed in FP64; the stress sum is FP64.
     * Each CTA holds its part's node state in shared memory: 96 bytes per
     * node for the FP32 kernel without its element table (velocity and
     * acceleration then live in global memory), which bounds an RVE to 16
     * parts of 2,186 nodes (34,976 nodes) on a GB300; a solve with a larger
     * RVE returns FE2_EINVAL (use FE2_PREC_FP64). */
    FE2_PREC_MIXED = 1
} fe2_precision;

typedef enum {
    FE2_INIT_REFERENCE = 0, /* free nodes start at u = 0 (only the fixed DOFs move) */
    FE2_INIT_AFFINE = 1,    /* every node starts at the affine position F X */
    FE2_INIT_WARM = 2       /* free nodes start at the batch's current displacement
                               (the last solve's result or fe2_batch_set_displacement) */
} fe2_init;

typedef struct {
    double tol;           /* relative residual tolerance, converged when
                             ||g_free||_2 <= tol * f_ref (default 1e-8) */
    int64_t max_iter;     /* iteration cap, >= 1 (default 10,000,000) */
    double dt_safety;     /* time-step safety factor alpha in (0, 1] (default 0.9) */
    int32_t precision;    /* fe2_precision (default FE2_PREC_MIXED) */
    int32_t init;         /* fe2_init (default FE2_INIT_AFFINE) */
    int32_t kinetic_energy; /* 1: also track the kinetic energy 1/2 sum m v^2;
                               2 (FE2_PREC_FP64 only): also the internal and
                               external work of the energy balance check
                               (fe2_batch_energy) */
    int32_t block_threads;  /* threads per CTA: 0 = default (512, the paper's
                               team size), else a multiple of 32 in [64, 512] */
    int64_t lead_iters;   /* MIXED: < 0 = lead until the relative residual
                             <= lead_tol (default); >= 0 = exactly that many
                             double-float iterations */
    int32_t rebase_every; /* MIXED: FP32 iterations between double-float
                             reference refreshes; <= 0 = default 512 */
    int32_t launch;       /* 0 = the batched solve replays a CUDA graph,
                             captured by the first solve with this option
                             set (default); 1 = plain stream launches */
    double lead_tol;      /* MIXED: relative residual that ends the lead
                             phase (default 1e-2) */
    int64_t stall_window; /* MIXED: FP32 evaluations in which the squared
                             residual must fall to a quarter of its reference
                             value; when it does not (the FP32 increments have
                             reached their rounding floor), the RVE is handed
                             back to a double-float resume that runs to
                             convergence. 0 = default 1,000,000; < 0 = never */
} fe2_opts;

/* Fill *opts with the defaults listed above. */
void fe2_opts_default(fe2_opts *opts);

/*
 * Launch tuning of the mixed solver per RVE size bucket b, the RVEs with
 * 2^b <= n_nodes < 2^(b+1): the cluster size (CTAs, i.e. spatial parts, per
 * RVE; a power of two <= 16) and the CTA sizes of the FP32 and lead kernels
 * (multiples of 32 in [64, 512]). Zero entries mean automatic: the smallest
 * cluster whose parts hold at most 1024 nodes, doubled while the FP32
 * kernel's element table does not fit in shared memory, and 512 threads.
 * The paper found the best team size to depend on the sub-problem size
 * (Section III); fe2_autotune measures it on this GPU.
 *
 * The setting is process-wide and applies to batches created, and plans
 * computed, after the call. A configuration is a function of the RVE's size
 * alone, so an RVE runs the same way in any batch; results change with it
 * only by rounding (the partition and the grouping of partial sums).
 */
typedef struct {
    int32_t parts[32];
    int32_t block_fp32[32];
    int32_t block_lead[32];
} fe2_tuning;

/* Set the process-wide tuning (NULL: every entry automatic). FE2_EINVAL for
 * an entry out of range; nothing changes then. */
fe2_status fe2_tuning_set(const fe2_tuning *t);
/* Copy the current tuning into *t. */
fe2_status fe2_tuning_get(fe2_tuning *t);
/* Set the tuning from a JSON file written by fe2_autotune. FE2_EINVAL if the
 * file cannot be read, is malformed, or was measured on another GPU model or
 * SM count. */
fe2_status fe2_tuning_load(const char *path);

/*
 * Autotuner of the mixed solver: for every size bucket present among the
 * given sample RVEs, time bounded solves (trial_iters iterations, a quarter of
 * them in the double-float lead) of the samples, replicated to fill the GPU,
 * for each feasible cluster size and FP32-kernel CTA size in {256, 384, 512},
 * and keep the pair with the most node-iterations per second per SM. The
 * result is set as the process-wide tuning, returned in *out (may be NULL)
 * and, if json_path is not NULL, written there as JSON keyed by GPU model,
 * SM count, precision and bucket. Inputs as for fe2_batch_create, plus F
 * (9*n_rve, row-major) for the trial solves. Synchronous; allocates and frees
 * its trial batches.
 */
fe2_status fe2_autotune(int32_t n_rve, const int64_t *node_off, const double *X,
                        const int64_t *elem_off, const int32_t *conn, const double *EA,
                        const uint8_t *fixed, const double *damping, const double *F,
                        int64_t trial_iters, const char *json_path, fe2_tuning *out);

/*
 * Create a batch of n_rve networks (Algorithm 1: load mesh, compute edge and
 * connectivity arrays, transfer them to the device, compute the lumped mass
 * matrix and the critical time step).
 *
 * n_rve     number of RVEs, >= 1.
 * node_off  n_rve+1 prefix offsets into the node arrays (node_off[0] = 0).
 * X         3*N reference coordinates, xyz interleaved, N = node_off[n_rve].
 * elem_off  n_rve+1 prefix offsets into the element arrays.
 * conn      2*E node ids, LOCAL to the element's RVE (0 .. n_p-1).
 * EA        E axial rigidities (> 0). The force law is N = EA (l/L - 1).
 * fixed     N flags: non-zero = prescribed displacement x = F X.
 * V0        n_rve reference volumes (> 0), or NULL for 1 (unit cube).
 * damping   n_rve damping coefficients c >= 0 (f_d = -c m v), or NULL for
 *           c = 0.002 (512 / n_p)^(1/3).
 * stream    cudaStream_t used for the uploads, or NULL (legacy stream).
 * out       receives the batch handle.
 *
 * Returns FE2_EINVAL if an id is out of range, an element joins a node to
 * itself or repeats another, a length is zero, EA <= 0, or a value is not
 * finite. A free node that no element touches is held fixed.
 */
fe2_status fe2_batch_create(int32_t n_rve, const int64_t *node_off, const double *X,
                            const int64_t *elem_off, const int32_t *conn, const double *EA,
                            const uint8_t *fixed, const double *V0, const double *damping,
                            void *stream, fe2_batch **out);

/*
 * Inspection call, host only (no device is touched): the packing that
 * fe2_batch_create computes for the same inputs (Algorithm 1: compute the
 * mesh connectivity array; Section III: the free/fixed reordering and the
 * packed CRS-style layout of many RVEs). It is the one call whose outputs
 * show the internal node order.
 *
 * Inputs as for fe2_batch_create. smem_optin is the device's opt-in shared
 * memory per block in bytes (it bounds the part size); nodes_per_cta is the
 * part-size target (<= 0: the default, as in fe2_batch_create).
 * Outputs (HOST, caller-allocated; each may be NULL):
 * parts     n_rve: CTAs (spatial parts) per RVE, a power of two <= 16.
 * perm      N: for each internal (permuted) node, the caller's global node
 *           index. Each RVE keeps its node range; within it, free nodes come
 *           first, part by part, then the fixed ones, part by part.
 * rowptr    N + n_rve: per RVE p, n_p + 1 CSR row offsets starting at
 *           node_off[p] + p, relative to the RVE's first entry.
 * col       2*E: per CSR entry, the neighbour's internal RVE-local index.
 *           Entries of a row follow the caller's neighbour ids.
 * col_part  2*E: the same neighbour as (part << 16 | index within its part).
 * part_off  n_rve * 34: per RVE, the first internal free node of each part
 *           (17 offsets), then the first fixed node of each part counted from
 *           the RVE's first fixed node (17 offsets).
 *
 * Returns FE2_EINVAL for the inputs fe2_batch_create rejects, or for
 * smem_optin <= 16384.
 */
fe2_status fe2_batch_layout(int32_t n_rve, const int64_t *node_off, const double *X,
                            const int64_t *elem_off, const int32_t *conn, const double *EA,
                            const uint8_t *fixed, int64_t smem_optin, int32_t nodes_per_cta,
                            int32_t *parts, int64_t *perm, int32_t *rowptr, int32_t *col,
                            int32_t *col_part, int32_t *part_off);

/*
 * Inspection call, host only: the element slot tables of the FP64 cluster
 * kernel for these inputs (Algorithm 1, getInternalForces on a cluster: each
 * CTA evaluates the elements with an end among its part's free nodes once per
 * iteration). Inputs as for fe2_batch_layout. Outputs (HOST, caller-allocated,
 * each may be NULL):
 * n_slots    total slots of the batch.
 * slot0      n_rve: the RVE's first slot.
 * part_slot  n_rve * 17: per RVE the parts' first slots relative to slot0
 *            (entry r+1 ends part r; entries past the RVE's parts repeat).
 * slot       4 per slot, at most cap slots: RVE-local element (caller
 *            numbering), its first and its second end as (part << 16 |
 *            index in the part's node order), 0.
 * csr_slot   2*E: per CSR entry (fe2_batch_layout's order) of a free node,
 *            its slot relative to its part's first << 1, | 1 when the node
 *            is the element's second end; -1 for entries of fixed nodes.
 * Returns FE2_EINVAL for the inputs fe2_batch_layout rejects.
 */
fe2_status fe2_batch_fp64_slots(int32_t n_rve, const int64_t *node_off, const double *X,
                                const int64_t *elem_off, const int32_t *conn, const double *EA,
                                const uint8_t *fixed, int64_t smem_optin, int32_t nodes_per_cta,
                                int64_t cap, int64_t *n_slots, int64_t *slot0, int32_t *part_slot,
                                int32_t *slot, int32_t *csr_slot);

/*
 * Inspection call, host only: the launch plan of the mixed solver
 * (FE2_PREC_MIXED) for these inputs, with the default CTA size. RVEs are
 * grouped into classes by cluster size and element-table staging; each class
 * runs three persistent launches (Algorithm 1's loop: the double-float lead,
 * the FP32 phase, and the double-float resume of RVEs whose FP32 residual
 * stalled) on a stream of its own.
 *
 * Inputs as for fe2_batch_layout. Outputs (HOST, caller-allocated; each may
 * be NULL); classes beyond max_classes are counted but not written:
 * n_classes    number of classes.
 * rve_class    n_rve: each RVE's class (index into the arrays below).
 * class_parts  per class: CTAs per cluster.
 * class_rves   per class: number of RVEs.
 * smem         2 per class: dynamic shared memory per CTA in bytes, for the
 *              lead kernel then for the FP32 kernel.
 * staged       2 per class (same order): 1 if that kernel keeps its
 *              element table in shared memory, 0 if it re-reads the CSR rows
 *              from global memory every iteration.
 * block        2 per class (same order): threads per CTA.
 *
 * Returns FE2_EINVAL for the inputs fe2_batch_layout rejects.
 */
fe2_status fe2_batch_plan(int32_t n_rve, const int64_t *node_off, const double *X,
                          const int64_t *elem_off, const int32_t *conn, const double *EA,
                          const uint8_t *fixed, int64_t smem_optin, int32_t nodes_per_cta,
                          int32_t max_classes, int32_t *n_classes, int32_t *rve_class,
                          int32_t *class_parts, int32_t *class_rves, int64_t *smem,
                          int32_t *staged, int32_t *block);

/*
 * Solve every RVE of the batch for its deformation gradient (Algorithm 1,
 * loop to convergence), asynchronously on `stream`.
 *
 * F     9*n_rve doubles, row-major, HOST memory (copied to the device on
 *       `stream` before the call returns).
 * opts  solver options, or NULL for fe2_opts_default().
 *
 * The RVEs run in persistent launches per size class (one for FP64; lead,
 * FP32 phase and resume for MIXED), the classes concurrently; the first solve
 * with an option set records them into a CUDA graph that later solves
 * replay (opts.launch). The host returns as soon as the work is queued.
 * Results are read with fe2_batch_stress() or fe2_batch_results_dev().
 */
fe2_status fe2_batch_solve(fe2_batch *b, const double *F, const fe2_opts *opts, void *stream);

/* As fe2_batch_solve(), with F already in DEVICE memory (9*n_rve doubles). */
fe2_status fe2_batch_solve_dev(fe2_batch *b, const double *F_dev, const fe2_opts *opts,
                               void *stream);

/*
 * Wait for the last solve and copy its results to HOST memory, indexed by RVE.
 * Any pointer may be NULL.
 *   sigma    9*n_rve volume-averaged Cauchy stress (1/V) sum_e (N_e/l_e) d_e d_e^T,
 *            V = det(F) V0, current configuration, row-major
 *   iters    n_rve iteration counts
 *   rel_res  n_rve final ||g_free|| / f_ref (0 when f_ref = 0)
 *   status   n_rve fe2_rve_status values
 * FE2_ESTATE before the first solve.
 */
fe2_status fe2_batch_stress(fe2_batch *b, double *sigma, int64_t *iters, double *rel_res,
                            int32_t *status);

/* Device-side results of the last solve, copied asynchronously on `stream`
 * into DEVICE buffers (any may be NULL). Same layouts as fe2_batch_stress(). */
fe2_status fe2_batch_results_dev(fe2_batch *b, double *sigma_dev, int64_t *iters_dev,
                                 double *rel_res_dev, int32_t *status_dev, void *stream);

/* Per-RVE diagnostics of the last batched solve (HOST memory, any may be
 * NULL): the residual scale f_ref = max(||g(F X)||, ||g(x0)||) over all DOFs,
 * the final kinetic energy (0 unless opts.kinetic_energy), and the number of
 * double-float lead iterations (MIXED; 0 for FP64). Waits for the solve. */
fe2_status fe2_batch_diagnostics(fe2_batch *b, double *f_ref, double *kinetic_energy,
                                 int64_t *lead_iters);

/*
 * Energy balance of the last batched solve (Algorithm 1, "optionally check
 * energy balance": three reductions over the free DOFs per iteration), per
 * RVE, HOST memory, any pointer may be NULL. Needs a last solve with
 * FE2_PREC_FP64 and opts.kinetic_energy = 2 (else FE2_ESTATE). With du the
 * step's displacement increment dt v^(n-1/2), g the net internal force and
 * f_d = -c m v^(n-1/2) the damping force, summed over free DOFs:
 *   kinetic        K = 1/2 sum m |v^n|^2 at the last iteration
 *   internal_work  Wint = -sum_steps 1/2 du . (g^(n-1) + g^n)  (stored energy)
 *   external_work  Wext =  sum_steps 1/2 du . (f_d^(n-1) + f_d^n) (damping,
 *                  <= 0; prescribed nodes do not move during the iteration)
 *   balance        (K + Wint - Wext) / max(|Wint|, |Wext|, K): the relative
 *                  balance error, nonzero by the time discretisation
 * Waits for the solve.
 */
fe2_status fe2_batch_energy(fe2_batch *b, double *kinetic, double *internal_work,
                            double *external_work, double *balance);

/* Cluster size (CTAs) the MIXED solver uses for each RVE (n_rve entries). */
fe2_status fe2_batch_parts(const fe2_batch *b, int32_t *parts);

/*
 * Serving: continuous micro-batching over the RVEs of one batch.
 *
 * In the FE2 scheme every macroscale step emits one microscale solve per
 * material point (Section I), and the paper's motivation is that this loop
 * runs millions of times per macroscale step (Section III). These calls let
 * a caller admit solves as they arrive instead of waiting for a whole batch.
 *
 * fe2_batch_submit: stage F for the n RVEs `rve_ids` (HOST arrays; 9*n
 * doubles row-major) and launch the solver for just those RVEs on a stream of
 * its own, returning at once. Submissions in flight overlap on the device. An
 * RVE keeps its state on the device, so opts->init = FE2_INIT_WARM restarts
 * from its last result. FE2_EBUSY when all 8 slots are in flight; FE2_EINVAL
 * if an id is out of range, repeated, or already in flight.
 *
 * fe2_batch_poll: hand back every finished submission that fits in `max`
 * entries: the RVE ids and, for each, sigma (9), iters, rel_res, status. Any
 * output pointer except n_out may be NULL. Never blocks.
 */
fe2_status fe2_batch_submit(fe2_batch *b, int32_t n, const int32_t *rve_ids, const double *F,
                            const fe2_opts *opts, int32_t *ticket);
fe2_status fe2_batch_poll(fe2_batch *b, int32_t max, int32_t *ids, double *sigma, int64_t *iters,
                          double *rel_res, int32_t *status, int32_t *n_out);

/*
 * A request loop over a timed schedule (synchronous; returns when every
 * request has completed). Request r asks for RVE rve[r] with deformation
 * gradient F[9r..9r+8], arriving at t_arrive[r] seconds after the call (non-
 * decreasing). A request becomes eligible once it has arrived and the previous
 * request of the same RVE has completed. Eligible requests are admitted in
 * micro-batches of at most max_batch RVEs (<= 0: no limit) while a serving
 * slot is free and the working set of the RVEs in flight stays within
 * max_inflight_bytes (<= 0: no limit). First solves of an RVE use opts_first;
 * later ones use opts_next (NULL: opts_first with FE2_INIT_WARM).
 * Outputs per request: t_done (seconds after the call, when its completion was
 * observed), and if non-NULL iters, status, sigma (9 per request).
 */
fe2_status fe2_serve(fe2_batch *b, int32_t n_req, const int32_t *rve, const double *t_arrive,
                     const double *F, const fe2_opts *opts_first, const fe2_opts *opts_next,
                     int32_t max_batch, double max_inflight_bytes, double *t_done, int64_t *iters,
                     int32_t *status, double *sigma);

/* Copy the current displacement u = x - X (3*N doubles, caller's node order
 * and numbering) to HOST memory. Waits for the last solve. */
fe2_status fe2_batch_get_displacement(fe2_batch *b, double *u);

/* Set the displacement used by the next FE2_INIT_WARM solve (3*N doubles,
 * HOST memory, caller's numbering). Fixed-node entries are ignored. */
fe2_status fe2_batch_set_displacement(fe2_batch *b, const double *u);

/* Release every resource of the batch. NULL is accepted. */
fe2_status fe2_batch_destroy(fe2_batch *b);

/* Batch facts: number of RVEs, total nodes, total elements, and the number
 * of kernel launches the last solve issued. Any pointer may be NULL. */
fe2_status fe2_batch_info(const fe2_batch *b, int32_t *n_rve, int64_t *n_nodes,
                          int64_t *n_elems, int32_t *launches);

/* Device time of each persistent launch of the last batched solve, measured
 * with CUDA events recorded on the stream that launched it (one entry per
 * size class; classes run concurrently). Waits for those launches.
 *   ms   out: up to `cap` durations in milliseconds
 *   n    out: number of timed launches (may exceed cap)
 * FE2_ESTATE before the first solve; after a naive solve *n = 0. */
fe2_status fe2_batch_kernel_times(fe2_batch *b, float *ms, int32_t cap, int32_t *n);

/*
 * The paper's naive path (Section III): the same FP64 algorithm solved one RVE
 * after another, each iteration as a short sequence of kernel launches
 * (fused free-DOF vector updates, zeroing plus an atomic scatter of the
 * element forces, and a residual reduction read back by the host every
 * iteration to test convergence). Kept as the comparator for the batched
 * path. Synchronous; results are read with fe2_batch_stress().
 */
fe2_status fe2_batch_solve_naive(fe2_batch *b, const double *F, const fe2_opts *opts,
                                 void *stream);

/*
 * Partition of a batch over n_ranks GPUs (Section I: every macroscale
 * material point's microscale problem is independent, so the batch shards
 * with no exchange during the iterations; only the 9-double stresses are
 * gathered afterwards). Host only. Longest processing time first: RVEs in
 * decreasing estimated cost, each to the least-loaded rank (ties: lower RVE
 * id first, lower rank). Cost = n_nodes * iters[p] when iters is given and
 * iters[p] > 0 (e.g. the previous solve's counts), else n_nodes^1.5 (the
 * iteration count of these networks grows about like n^0.5).
 * node_off  n_rve+1 prefix offsets (as in fe2_batch_create)
 * iters     n_rve iteration counts, or NULL
 * rank_of   out: n_rve rank of each RVE
 * rank_cost out (may be NULL): n_ranks summed cost per rank
 */
fe2_status fe2_shard_plan(int32_t n_rve, const int64_t *node_off, const int64_t *iters,
                          int32_t n_ranks, int32_t *rank_of, double *rank_cost);

/* Message of the last failed call on this thread ("" if none). */
const char *fe2_last_error(void);

/*
 * Allocation-free solve of ONE RVE. The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc (code running during
 * CUDA graph capture, real-time loops that must not allocate, frameworks that
 * own every device allocation through their own pools). It allocates nothing:
 * inputs and outputs are the caller's DEVICE buffers, and all working memory
 * is one file-scope device array of fe2_noalloc_scratch_bytes() bytes (about
 * 1.6 MB) that every GPU loading the library holds until the process exits.
 *
 * It runs the same per-RVE FP64 solver as fe2_batch_solve with
 * FE2_PREC_FP64, in one CTA. Every node's update is the same sequence of IEEE
 * operations as on that path, but the free nodes are held in the caller's
 * order rather than the batch's spatial order, so the residual sum is
 * associated differently: rel_res agrees with the batched path to about
 * 1e-12, and where the two iteration counts agree (they can differ by one
 * when the residual lands within rounding of the threshold) the
 * displacement is bit-identical and sigma agrees to about 1e-12.
 *
 * n_nodes    1 .. 4096 nodes;  n_elems  0 .. 16384 elements (else FE2_EINVAL)
 * X_dev      3*n_nodes reference coordinates, xyz interleaved
 * conn_dev   2*n_elems node ids (0 .. n_nodes-1);  EA_dev  n_elems rigidities
 * fixed_dev  n_nodes flags (non-zero: prescribed x = F X)
 * F_dev      9 doubles, row-major
 * damping    c >= 0, or negative for 0.002 (512/n)^(1/3);  V0 > 0
 * opts       as for fe2_batch_solve; precision must be FE2_PREC_FP64
 * u_dev      3*n_nodes: read for FE2_INIT_WARM (free nodes), written with
 *            the final displacement (caller's node order)
 * sigma_dev (9), iters_dev (1), rel_res_dev (1), status_dev (1): outputs;
 *            status 4 means the device-side input checks failed (an id out of
 *            range, a self-loop, a repeated element, a zero length, EA <= 0 or
 *            a non-finite value) and nothing was solved.
 * stream     cudaStream_t or NULL. The call is asynchronous on it.
 *
 * The scratch array is shared by all calls on a device and keeps the last
 * call's contents; each solve rewrites or clears everything it reads. Calls
 * whose work overlaps on the GPU (other streams, other host threads) race on
 * it: serialise them. The first call on a device looks up the array's device
 * address (and sets the kernel's shared-memory limit); make that first call
 * before any stream capture.
 */
fe2_status fe2_rve_solve_noalloc(int32_t n_nodes, int32_t n_elems, const double *X_dev,
                                 const int32_t *conn_dev, const double *EA_dev,
                                 const uint8_t *fixed_dev, const double *F_dev, double damping,
                                 double V0, const fe2_opts *opts, double *u_dev, double *sigma_dev,
                                 int64_t *iters_dev, double *rel_res_dev, int32_t *status_dev,
                                 void *stream);

/* Size in bytes of the allocation-free entry point's device scratch array. */
size_t fe2_noalloc_scratch_bytes(void);

/* Message of the last failed fe2_rve_solve_noalloc call on this thread. */
const char *fe2_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FE2_H */
