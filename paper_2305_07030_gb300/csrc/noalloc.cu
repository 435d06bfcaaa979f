// Allocation-free single-RVE solve: the FP64 oracle-order solver with all of
// its working memory in one file-scope device array.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured, real-time loops that must not allocate, or host frameworks
// that own every device allocation through their own pools. They hold their
// inputs and outputs in device memory they already have and need the library
// to allocate nothing. fe2_rve_solve_noalloc serves them: it packs one RVE into
// the static scratch array below (node permutation, node-centric CSR, lumped
// masses, critical time step) and runs the same per-RVE FP64 solver as the
// batched FP64 path, inside a single CTA.
//
// The scratch array is shared by every call on a device and keeps the last
// call's contents; everything a solve reads is rewritten or cleared by that
// solve. Calls whose work overlaps on the GPU race on it. The array occupies
// kNoallocScratchBytes of device memory on every GPU that loads the library,
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/fe2.h"
#include "dr_fp64.cuh"

namespace fe2 {
namespace {

constexpr int kNaMaxNodes = 4096;
constexpr int kNaMaxElems = 16384;
constexpr int kNaThreads = 512;

// Byte layout of the scratch array (every block 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffRve = 0;
constexpr size_t kOffX = align256(kOffRve + sizeof(RveDesc));
constexpr size_t kOffMass = align256(kOffX + sizeof(double) * 3 * kNaMaxNodes);
constexpr size_t kOffU = align256(kOffMass + sizeof(double) * kNaMaxNodes);
constexpr size_t kOffV = align256(kOffU + sizeof(double) * 3 * kNaMaxNodes);
constexpr size_t kOffA = align256(kOffV + sizeof(double) * 3 * kNaMaxNodes);
constexpr size_t kOffRow = align256(kOffA + sizeof(double) * 3 * kNaMaxNodes);
constexpr size_t kOffCol = align256(kOffRow + sizeof(int32_t) * (kNaMaxNodes + 1));
constexpr size_t kOffElemOf = align256(kOffCol + sizeof(int32_t) * 2 * kNaMaxElems);
constexpr size_t kOffEAc = align256(kOffElemOf + sizeof(int32_t) * 2 * kNaMaxElems);
constexpr size_t kOffLc = align256(kOffEAc + sizeof(double) * 2 * kNaMaxElems);
constexpr size_t kOffElA = align256(kOffLc + sizeof(double) * 2 * kNaMaxElems);
constexpr size_t kOffElB = align256(kOffElA + sizeof(int32_t) * kNaMaxElems);
constexpr size_t kOffElEA = align256(kOffElB + sizeof(int32_t) * kNaMaxElems);
constexpr size_t kOffElL = align256(kOffElEA + sizeof(double) * kNaMaxElems);
constexpr size_t kOffPerm = align256(kOffElL + sizeof(double) * kNaMaxElems);  // permuted -> caller
constexpr size_t kOffInv = align256(kOffPerm + sizeof(int32_t) * kNaMaxNodes);  // caller -> permuted
constexpr size_t kOffDeg = align256(kOffInv + sizeof(int32_t) * kNaMaxNodes);
constexpr size_t kOffCur = align256(kOffDeg + sizeof(int32_t) * kNaMaxNodes);
constexpr size_t kOffMisc = align256(kOffCur + sizeof(int32_t) * kNaMaxNodes);  // f_ref, ke
constexpr size_t kNoallocScratchBytes = align256(kOffMisc + 2 * sizeof(double));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Per-RVE status written when the device-side input checks fail.
constexpr int kRveInvalid = 4;

struct NaArgs {
    int n, E;
    const double *X;       // caller, 3n xyz interleaved
    const int32_t *conn;   // caller, 2E local ids
    const double *EA;      // caller, E
    const uint8_t *fixed;  // caller, n
    const double *F;       // caller, 9
    double c, V0;
    double *u;             // caller, 3n (input for warm start, output)
    double *sigma;         // caller, 9
    int64_t *iters;        // caller, 1
    double *rel_res;       // caller, 1
    int32_t *status;       // caller, 1
};

__device__ __forceinline__ int block_excl_scan(int v, int *tmp) {
    // exclusive scan over the CTA (kNaThreads threads, 16 warps)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (kNaThreads >> 5) ? tmp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (kNaThreads >> 5)) tmp[lane] = w;
    }
    __syncthreads();
    const int before = warp > 0 ? tmp[warp - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kNaThreads) k_noalloc_solve(NaArgs A, SolveParams P, unsigned char *scr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[32];
    __shared__ int tmp[32];
    __shared__ int err, nfree_s;
    RveDesc *rve = reinterpret_cast<RveDesc *>(scr + kOffRve);
    double *X = reinterpret_cast<double *>(scr + kOffX);
    double *mass = reinterpret_cast<double *>(scr + kOffMass);
    double *u = reinterpret_cast<double *>(scr + kOffU);
    double *v = reinterpret_cast<double *>(scr + kOffV);
    double *a = reinterpret_cast<double *>(scr + kOffA);
    int32_t *row = reinterpret_cast<int32_t *>(scr + kOffRow);
    int32_t *col = reinterpret_cast<int32_t *>(scr + kOffCol);
    int32_t *elem_of = reinterpret_cast<int32_t *>(scr + kOffElemOf);
    double *EAc = reinterpret_cast<double *>(scr + kOffEAc);
    double *Lc = reinterpret_cast<double *>(scr + kOffLc);
    int32_t *el_a = reinterpret_cast<int32_t *>(scr + kOffElA);
    int32_t *el_b = reinterpret_cast<int32_t *>(scr + kOffElB);
    double *el_EA = reinterpret_cast<double *>(scr + kOffElEA);
    double *el_L = reinterpret_cast<double *>(scr + kOffElL);
    int32_t *perm = reinterpret_cast<int32_t *>(scr + kOffPerm);
    int32_t *inv = reinterpret_cast<int32_t *>(scr + kOffInv);
    int32_t *deg = reinterpret_cast<int32_t *>(scr + kOffDeg);
    int32_t *cur = reinterpret_cast<int32_t *>(scr + kOffCur);
    double *misc = reinterpret_cast<double *>(scr + kOffMisc);
    const int n = A.n, E = A.E;

    // ---- checks of the device-side inputs; degrees ----
    if (threadIdx.x == 0) err = 0;
    __syncthreads();  // the flag is clear before any thread may set it
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        deg[i] = 0;
        const double *x = A.X + 3 * i;
        if (!isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2])) err = 1;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int p = A.conn[2 * e], q = A.conn[2 * e + 1];
        if (p < 0 || q < 0 || p >= n || q >= n || p == q || !(A.EA[e] > 0.0) || !isfinite(A.EA[e])) {
            err = 1;
            continue;
        }
        const double *xp = A.X + 3 * p, *xq = A.X + 3 * q;
        if (xp[0] == xq[0] && xp[1] == xq[1] && xp[2] == xq[2]) err = 1;
        atomicAdd(deg + p, 1);
        atomicAdd(deg + q, 1);
    }
    __syncthreads();
    if (err) {
        if (threadIdx.x == 0) {
            *A.status = kRveInvalid;
            *A.iters = 0;
            *A.rel_res = 0.0;
        }
        return;
    }

    // ---- permutation: free nodes first, then fixed, each in caller order ----
    // (a free node that no element touches is held fixed)
    constexpr int kPer = kNaMaxNodes / kNaThreads;
    int fl[kPer], cnt = 0;
    for (int k = 0; k < kPer; ++k) {
        const int i = threadIdx.x * kPer + k;
        fl[k] = (i < n && !A.fixed[i] && deg[i] > 0) ? 1 : 0;
        cnt += fl[k];
    }
    int off = block_excl_scan(cnt, tmp);
    if (threadIdx.x == blockDim.x - 1) nfree_s = off + cnt;
    __syncthreads();
    const int nf = nfree_s;
    int offx = block_excl_scan((threadIdx.x * kPer < n ? min(kPer, n - (int)threadIdx.x * kPer) : 0) - cnt, tmp);
    for (int k = 0; k < kPer; ++k) {
        const int i = threadIdx.x * kPer + k;
        if (i >= n) break;
        const int pi = fl[k] ? off++ : nf + offx++;
        perm[pi] = i;
        inv[i] = pi;
    }
    __syncthreads();

    // ---- node-centric CSR: row pointers, entries, rows sorted by caller id ----
    int dsum = 0;
    for (int k = 0; k < kPer; ++k) {
        const int pi = threadIdx.x * kPer + k;
        if (pi < n) dsum += deg[perm[pi]];
    }
    int roff = block_excl_scan(dsum, tmp);
    for (int k = 0; k < kPer; ++k) {
        const int pi = threadIdx.x * kPer + k;
        if (pi < n) {
            row[pi] = roff;
            cur[pi] = roff;
            roff += deg[perm[pi]];
        }
    }
    if (threadIdx.x == 0) row[n] = 2 * E;
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int p = inv[A.conn[2 * e]], q = inv[A.conn[2 * e + 1]];
        const int sp = atomicAdd(cur + p, 1), sq = atomicAdd(cur + q, 1);
        col[sp] = q; elem_of[sp] = e;
        col[sq] = p; elem_of[sq] = e;
    }
    __syncthreads();
    for (int pi = threadIdx.x; pi < n; pi += blockDim.x) {
        const int b = row[pi], en = row[pi + 1];
        for (int s = b + 1; s < en; ++s) {  // insertion sort by caller id of the neighbour
            const int cj = col[s], ej = elem_of[s], key = perm[cj];
            int t = s - 1;
            while (t >= b && perm[col[t]] > key) {
                col[t + 1] = col[t];
                elem_of[t + 1] = elem_of[t];
                --t;
            }
            col[t + 1] = cj;
            elem_of[t + 1] = ej;
        }
        for (int s = b + 1; s < en; ++s)
            if (col[s] == col[s - 1]) err = 1;  // repeated element
    }
    __syncthreads();
    if (err) {
        if (threadIdx.x == 0) {
            *A.status = kRveInvalid;
            *A.iters = 0;
            *A.rel_res = 0.0;
        }
        return;
    }

    // ---- coordinates, lengths, masses, stress elements, time step ----
    for (int pi = threadIdx.x; pi < n; pi += blockDim.x) {
        const int i = perm[pi];
        for (int c = 0; c < 3; ++c) X[c * n + pi] = A.X[3 * i + c];
    }
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const int p = A.conn[2 * e], q = A.conn[2 * e + 1];
        const double *xp = A.X + 3 * p, *xq = A.X + 3 * q;
        const double dx = dsub(xq[0], xp[0]), dy = dsub(xq[1], xp[1]), dz = dsub(xq[2], xp[2]);
        el_L[e] = dsqrt(dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)));
        el_a[e] = inv[p];
        el_b[e] = inv[q];
        el_EA[e] = A.EA[e];
    }
    __syncthreads();
    for (int s = threadIdx.x; s < 2 * E; s += blockDim.x) {
        EAc[s] = A.EA[elem_of[s]];
        Lc[s] = el_L[elem_of[s]];
    }
    __syncthreads();
    for (int pi = threadIdx.x; pi < n; pi += blockDim.x) {
        double m = 0.0;
        for (int s = row[pi]; s < row[pi + 1]; ++s) {
            const double L = Lc[s];
            const double rhoA = ddiv(EAc[s], dmul(L, L));
            m = dadd(m, dmul(0.5, dmul(rhoA, L)));
        }
        mass[pi] = m;
        // warm start reads the caller's displacement (caller order)
        for (int c = 0; c < 3; ++c) u[c * n + pi] = P.init == 2 ? A.u[3 * perm[pi] + c] : 0.0;
    }
    double tmin = INFINITY;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        const double L = el_L[e], EA = el_EA[e];
        const double rhoA = ddiv(EA, dmul(L, L));
        const double t = dmul(L, dsqrt(ddiv(rhoA, EA)));
        tmin = t < tmin ? t : tmin;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_xor_sync(0xffffffffu, tmin, o);
        tmin = other < tmin ? other : tmin;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tmin;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = INFINITY;
        for (int w = 0; w < (kNaThreads >> 5); ++w) t = red[w] < t ? red[w] : t;
        RveDesc R;
        R.node0 = 0; R.rp0 = 0; R.csr0 = 0; R.elem0 = 0;
        R.n_nodes = n; R.n_free = nf; R.n_elems = E; R.n_parts = 1;
        R.dtc = t; R.c = A.c; R.V0 = A.V0; R.part_max = n; R.part_free_max = nf;
        R.part_elem_max = 0; R.part_slot_max = 0;
        *rve = R;
    }
    __syncthreads();

    // ---- the solve: the batched FP64 path's per-RVE solver ----
    DevMesh M = {};
    M.rve = rve;
    M.X0 = X; M.X1 = X + n; M.X2 = X + 2 * n;
    M.mass = mass;
    M.rowptr = row;
    M.col = col;
    M.EA = EAc;
    M.L = Lc;
    M.el_a = el_a; M.el_b = el_b; M.el_EA = el_EA; M.el_L = el_L;
    DevState S = {};
    S.u0 = u; S.u1 = u + n; S.u2 = u + 2 * n;
    S.v0 = v; S.v1 = v + n; S.v2 = v + 2 * n;
    S.a0 = a; S.a1 = a + n; S.a2 = a + 2 * n;
    DevResults O = {};
    O.sigma = A.sigma; O.iters = A.iters; O.rel_res = A.rel_res; O.status = A.status;
    O.f_ref = misc; O.ke = misc + 1;
    solve_rve_fp64<true, false>(M, S, O, P, 0, reinterpret_cast<double *>(smem_raw), red);

    // ---- displacement back in the caller's order ----
    for (int pi = threadIdx.x; pi < n; pi += blockDim.x) {
        const int i = perm[pi];
        for (int c = 0; c < 3; ++c) A.u[3 * i + c] = u[c * n + pi];
    }
}

std::mutex g_na_mutex;
void *g_na_ptr[64] = {};
bool g_na_attr[64] = {};
thread_local std::string g_na_err;

}  // namespace
}  // namespace fe2

using namespace fe2;

extern "C" const char *fe2_noalloc_last_error(void) { return g_na_err.c_str(); }

extern "C" size_t fe2_noalloc_scratch_bytes(void) { return kNoallocScratchBytes; }

extern "C" fe2_status fe2_rve_solve_noalloc(int32_t n_nodes, int32_t n_elems, const double *X_dev,
                                            const int32_t *conn_dev, const double *EA_dev,
                                            const uint8_t *fixed_dev, const double *F_dev,
                                            double damping, double V0, const fe2_opts *opts,
                                            double *u_dev, double *sigma_dev, int64_t *iters_dev,
                                            double *rel_res_dev, int32_t *status_dev,
                                            void *stream) {
    if (n_nodes < 1 || n_nodes > kNaMaxNodes) {
        g_na_err = "n_nodes must be in [1, " + std::to_string(kNaMaxNodes) + "]";
        return FE2_EINVAL;
    }
    if (n_elems < 0 || n_elems > kNaMaxElems) {
        g_na_err = "n_elems must be in [0, " + std::to_string(kNaMaxElems) + "]";
        return FE2_EINVAL;
    }
    if (!X_dev || !fixed_dev || !F_dev || !u_dev || !sigma_dev || !iters_dev || !rel_res_dev ||
        !status_dev || (n_elems > 0 && (!conn_dev || !EA_dev))) {
        g_na_err = "NULL device pointer";
        return FE2_EINVAL;
    }
    fe2_opts o;
    if (opts) o = *opts; else fe2_opts_default(&o);
    if (o.precision != FE2_PREC_FP64) {
        g_na_err = "the allocation-free entry point runs the FP64 solver only";
        return FE2_EINVAL;
    }
    if (!(o.tol >= 0.0) || o.max_iter < 1 || !(o.dt_safety > 0.0 && o.dt_safety <= 1.0) ||
        o.init < 0 || o.init > 2) {
        g_na_err = "invalid options";
        return FE2_EINVAL;
    }
    if (!(V0 > 0.0)) {
        g_na_err = "V0 must be > 0";
        return FE2_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        g_na_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return FE2_ECUDA;
    }
    void *scratch = nullptr;
    {
        // once per device, with that device current: the device address of the
        // scratch array (its name in host code is not a device address)
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            e = cudaGetSymbolAddress(&g_na_ptr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_na_ptr[dev] = nullptr;
                g_na_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
                return FE2_ECUDA;
            }
        }
        if (!g_na_attr[dev]) {
            e = cudaFuncSetAttribute(k_noalloc_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(double) * 3 * kNaMaxNodes));
            if (e != cudaSuccess) {
                g_na_err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
                return FE2_ECUDA;
            }
            g_na_attr[dev] = true;
        }
        scratch = g_na_ptr[dev];
    }
    NaArgs A;
    A.n = n_nodes;
    A.E = n_elems;
    A.X = X_dev;
    A.conn = conn_dev;
    A.EA = EA_dev;
    A.fixed = fixed_dev;
    A.F = F_dev;
    A.c = damping >= 0.0 ? damping : 0.002 * cbrt(512.0 / (double)n_nodes);
    A.V0 = V0;
    A.u = u_dev;
    A.sigma = sigma_dev;
    A.iters = iters_dev;
    A.rel_res = rel_res_dev;
    A.status = status_dev;
    SolveParams P = {};
    P.F = F_dev;
    P.tol = o.tol;
    P.max_iter = o.max_iter;
    P.alpha = o.dt_safety;
    P.init = o.init;
    P.want_ke = o.kinetic_energy != 0 ? 1 : 0;  // kinetic energy only: no work-sum scratch here
    P.lead_iters = -1;
    P.lead_tol = 0.0;
    P.smem_positions = 1;
    const size_t smem = sizeof(double) * 3 * (size_t)n_nodes;
    k_noalloc_solve<<<1, kNaThreads, smem, static_cast<cudaStream_t>(stream)>>>(
        A, P, static_cast<unsigned char *>(scratch));
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_na_err = std::string("launch: ") + cudaGetErrorString(e);
        return FE2_ECUDA;
    }
    return FE2_OK;
}
