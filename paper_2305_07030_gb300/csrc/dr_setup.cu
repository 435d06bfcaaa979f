// Create-time kernels (Algorithm 1: reference lengths, lumped mass matrix by
// element integration, critical time step). Run once per batch.
#include "dr_device.cuh"

namespace fe2 {

// L_e = |X_b - X_a| for every element (a, b global permuted node ids, oriented
// as the caller's a < b).
__global__ void k_elem_lengths(int64_t n_el, const int64_t *ga, const int64_t *gb,
                               const double *X0, const double *X1, const double *X2,
                               double *L) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n_el;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = ga[e], b = gb[e];
        const double dx = dsub(X0[b], X0[a]), dy = dsub(X1[b], X1[a]), dz = dsub(X2[b], X2[a]);
        L[e] = dsqrt(dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)));
    }
}

__device__ __forceinline__ void split_df(double d, float &hi, float &lo) {
    hi = __double2float_rn(d);
    lo = __double2float_rn(d - (double)hi);
}

// Per CSR entry: the element's L, and (EA, 1/L) as double-float pairs.
__global__ void k_csr_fill(int64_t n_csr, const int64_t *elem_of, const double *el_L,
                           const double *EA_csr, double *L_csr, float2 *eaf, float2 *eaf_lo) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n_csr;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double L = el_L[elem_of[k]];
        L_csr[k] = L;
        float eh, el, ih, il;
        split_df(EA_csr[k], eh, el);
        split_df(1.0 / L, ih, il);
        eaf[k] = make_float2(eh, ih);
        eaf_lo[k] = make_float2(el, il);
    }
}

// One CTA per RVE: lumped masses m_i = sum_e 1/2 rho A_e L_e with
// rho A_e = EA_e / L_e^2 (in the node's element order), and the critical step
// min_e L_e sqrt(rho A_e / EA_e).
__global__ void k_mass_dt(RveDesc *rve, const int32_t *rowptr, const int32_t *col,
                          const double *EA_csr, const double *L_csr, const double *el_EA,
                          const double *el_L, const double *X0, const double *X1,
                          const double *X2, double *mass, float *imh, float *iml, float *Xh,
                          float *Xl, float4 *dh, float4 *dl) {
    __shared__ double red[32];
    RveDesc &R = rve[blockIdx.x];
    const int32_t *rp = rowptr + R.rp0;
    for (int i = threadIdx.x; i < R.n_nodes; i += blockDim.x) {
        double m = 0.0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int64_t kk = R.csr0 + k;
            const double L = L_csr[kk];
            const double rhoA = ddiv(EA_csr[kk], dmul(L, L));
            m = dadd(m, dmul(0.5, dmul(rhoA, L)));
        }
        // per CSR entry: D = X_j - X_i and the reference length, double-float
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int64_t kk = R.csr0 + k;
            const int64_t j = R.node0 + col[kk], ii = R.node0 + i;
            float a0, b0, a1, b1, a2, b2, a3, b3;
            split_df(dsub(X0[j], X0[ii]), a0, b0);
            split_df(dsub(X1[j], X1[ii]), a1, b1);
            split_df(dsub(X2[j], X2[ii]), a2, b2);
            split_df(L_csr[kk], a3, b3);
            dh[kk] = make_float4(a0, a1, a2, a3);
            dl[kk] = make_float4(b0, b1, b2, b3);
        }
        mass[R.node0 + i] = m;
        float h = 0.f, l = 0.f;
        if (m > 0.0) split_df(1.0 / m, h, l);
        imh[R.node0 + i] = h;
        iml[R.node0 + i] = l;
        // reference coordinates as double-float, per-RVE [3][n] blocks
        const double X[3] = {X0[R.node0 + i], X1[R.node0 + i], X2[R.node0 + i]};
        for (int c = 0; c < 3; ++c)
            split_df(X[c], Xh[3 * R.node0 + c * R.n_nodes + i], Xl[3 * R.node0 + c * R.n_nodes + i]);
    }
    double tmin = INFINITY;
    for (int e = threadIdx.x; e < R.n_elems; e += blockDim.x) {
        const int64_t ee = R.elem0 + e;
        const double L = el_L[ee], EA = el_EA[ee];
        const double rhoA = ddiv(EA, dmul(L, L));
        const double t = dmul(L, dsqrt(ddiv(rhoA, EA)));
        tmin = t < tmin ? t : tmin;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_xor_sync(0xffffffffu, tmin, o);
        tmin = other < tmin ? other : tmin;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = tmin;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = INFINITY;
        for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t = red[w] < t ? red[w] : t;
        R.dtc = t;
    }
}

int launch_setup(int32_t n_rve, int64_t n_el, int64_t n_csr, RveDesc *rve,
                 const int64_t *ga, const int64_t *gb, const double *X0, const double *X1,
                 const double *X2, const int64_t *elem_of, const double *EA_csr,
                 const double *el_EA, const int32_t *rowptr, double *el_L, double *L_csr,
                 float2 *eaf, float2 *eaf_lo, double *mass, float *imh, float *iml,
                 float *Xh, float *Xl, const int32_t *col, float4 *dh, float4 *dl,
                 void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (n_el > 0) {
        const int g = (int)((n_el + 255) / 256 < 65535 ? (n_el + 255) / 256 : 65535);
        k_elem_lengths<<<g, 256, 0, st>>>(n_el, ga, gb, X0, X1, X2, el_L);
    }
    if (n_csr > 0) {
        const int g = (int)((n_csr + 255) / 256 < 65535 ? (n_csr + 255) / 256 : 65535);
        k_csr_fill<<<g, 256, 0, st>>>(n_csr, elem_of, el_L, EA_csr, L_csr, eaf, eaf_lo);
    }
    k_mass_dt<<<n_rve, 256, 0, st>>>(rve, rowptr, col, EA_csr, L_csr, el_EA, el_L, X0, X1, X2,
                                     mass, imh, iml, Xh, Xl, dh, dl);
    return (int)cudaGetLastError();
}

}  // namespace fe2
