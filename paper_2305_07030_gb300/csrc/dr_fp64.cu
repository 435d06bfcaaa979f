// FP64 dynamic relaxation (Algorithm 1) for a batch of RVEs: one CTA per RVE,
// whole loop inside one persistent launch.
//
// The paper moved the entire relaxation loop into one kernel with one thread
// team per sub-problem to remove the per-iteration launch overhead
// (Section III). Here a persistent grid pops RVEs from a cost-ordered work
// queue; each CTA stages the RVE's current positions in shared memory (or in
// an L2-resident scratch when they do not fit), evaluates each element's
// force once into an L2-resident table and sums it per node in the node's
// row order (no atomics), and keeps the loop scalars (iteration count, residual)
// CTA-uniform so that every thread takes the same exit.
//
// Arithmetic is IEEE FP64 with explicit rounding in the order of a serial
// element-scatter implementation, so the trajectory is bit-identical to one
// (only the residual and stress sums are reassociated).
#include "dr_fp64.cuh"

namespace fe2 {

template <bool SM>
__global__ void __launch_bounds__(512) dr_fp64_kernel(DevMesh M, DevState S, DevResults O,
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
        solve_rve_fp64<SM, true>(M, S, O, P, P.queue[item], reinterpret_cast<double *>(smem_raw), red);
    }
}

namespace {
// Raise the staged kernel's shared-memory limit once per device and size (no
// attribute call while a launch is recorded into a CUDA graph).
void prepare_fp64(size_t smem) {
    static int set_bytes[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || set_bytes[dev] < (int)smem) {
        cudaFuncSetAttribute(dr_fp64_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (dev >= 0 && dev < 64) set_bytes[dev] = (int)smem;
    }
}
}  // namespace

int launch_dr_fp64(const DevMesh &m, const DevState &s, const DevResults &r, const SolveParams &p,
                   int grid, int block, size_t smem, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (p.smem_positions) {
        prepare_fp64(smem);
        dr_fp64_kernel<true><<<grid, block, smem, st>>>(m, s, r, p);
    } else {
        dr_fp64_kernel<false><<<grid, block, 0, st>>>(m, s, r, p);
    }
    return (int)cudaGetLastError();
}

int occupancy_dr_fp64(int smem_positions, int block, size_t smem) {
    int n = 0;
    if (smem_positions) {
        prepare_fp64(smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dr_fp64_kernel<true>, block, smem);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, dr_fp64_kernel<false>, block, 0);
    }
    return n;
}

}  // namespace fe2
