// Hand-written adjoint of the damped Euler-Cromer run with frozen bond flags
// (FP64).  One reverse step n+1 -> n is two launches:
//   k_adj_mask  w = ws (vbar + dt ubar) with the controlled components of ubar
//               and vbar zeroed (a prescribed component does not depend on the
//               previous state); ws = 1 for an Euler-Cromer step, 1/2 for the
//               half kicks that open and close a velocity-Verlet run
//   k_adj_step  per node m over its family (the same sliced layout and lane-per-
//               node walk as the forward step):
//                 ubar^n_m = ubar_m + (dt/rho) sum_j c_mj K_mj (V_m w_j - V_j w_m)
//                 vbar^n_m = (1 - dt eta/rho) w_m
//               with K = (1/L - 1/r) I + y y^T / r^3, the derivative of s y/|y|
//               (Eqs. 4-5) with respect to y = xi + eta; it also accumulates the
//               gradient of every directed bond's stiffness,
//                 dL/dc[m->j] += (dt/rho) s V_j (y/r).w_m
//               and the node's load sensitivity force_m . w_m.
// The stiffness of a bond is symmetric (c_mj = c_jm), as the forward requires.
#include <cuda_runtime.h>

#include <algorithm>

#include "pd_internal.h"

namespace pd {
namespace {

#define GRID_STRIDE(var, count)                                                   \
    for (int64_t var = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; var < (count); \
         var += (int64_t)gridDim.x * blockDim.x)

int grid_for(int64_t work, int block)
{
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 65535 * 8) g = 65535 * 8;
    return (int)g;
}

__global__ void k_adj_mask(const double* __restrict__ ub, const double* __restrict__ vb,
                           const uint8_t* __restrict__ bcc, const BcClass* __restrict__ bct,
                           int64_t n, double dt, double ws, double* __restrict__ ubm,
                           double* __restrict__ w)
{
    GRID_STRIDE(p, n)
    {
        const uint32_t cls = bcc[p];
        const uint32_t mask = cls ? bct[cls].mask : 0u;
        for (int c = 0; c < 3; ++c) {
            const bool ctl = (mask >> c) & 1u;
            const double u = ctl ? 0.0 : ub[3 * p + c];
            const double v = ctl ? 0.0 : vb[3 * p + c];
            ubm[3 * p + c] = u;
            w[3 * p + c] = ws * (v + dt * u);
        }
    }
}

__global__ void __launch_bounds__(256) k_adj_step(const AdjArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int Q = a.Q;
    const int64_t W = 32LL * Q;
    const int64_t nslices = (a.n + 31) >> 5;
    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int64_t m = (g << 5) + lane;
        const int Wg = a.sw[g];
        const double xm0 = a.x64[3 * m], xm1 = a.x64[3 * m + 1], xm2 = a.x64[3 * m + 2];
        const double um0 = a.un[3 * m], um1 = a.un[3 * m + 1], um2 = a.un[3 * m + 2];
        const double wm0 = a.w[3 * m], wm1 = a.w[3 * m + 1], wm2 = a.w[3 * m + 2];
        const double Vm = a.vol[m];
        double acc0 = 0.0, acc1 = 0.0, acc2 = 0.0;
        for (int q = 0; q * 32 < Wg; ++q) {
            const uint32_t word = a.bits[(g * Q + q) * 32 + lane];
            const int mend = min(32, Wg - q * 32);
            for (int b = 0; b < mend; ++b) {
                if (!((word >> b) & 1u)) continue;
                const int64_t slot = (g * W + q * 32 + b) * 32 + lane;
                const int64_t j = a.nbr[slot];
                const double e0 = a.x64[3 * j] - xm0, e1 = a.x64[3 * j + 1] - xm1,
                             e2 = a.x64[3 * j + 2] - xm2;
                const double y0 = e0 + (a.un[3 * j] - um0), y1 = e1 + (a.un[3 * j + 1] - um1),
                             y2 = e2 + (a.un[3 * j + 2] - um2);
                const double iL = a.ilen[slot];
                const double yy2 = y0 * y0 + y1 * y1 + y2 * y2;
                const double ir = rsqrt_nr(yy2);
                const double r = yy2 * ir;
                const double s = fma(r, iL, -1.0);
                const double Vj = a.vol[j];
                const double d0 = Vm * a.w[3 * j] - Vj * wm0;
                const double d1 = Vm * a.w[3 * j + 1] - Vj * wm1;
                const double d2 = Vm * a.w[3 * j + 2] - Vj * wm2;
                const double yd = y0 * d0 + y1 * d1 + y2 * d2;
                const double cij = a.cbond != nullptr ? a.cbond[slot] : a.c;
                const double k1 = iL - ir, k2 = yd * (ir * ir * ir);
                acc0 += cij * (k1 * d0 + y0 * k2);
                acc1 += cij * (k1 * d1 + y1 * k2);
                acc2 += cij * (k1 * d2 + y2 * k2);
                const double yw = y0 * wm0 + y1 * wm1 + y2 * wm2;
                a.gc[slot] += a.dt_rho * s * Vj * yw * ir;
            }
        }
        if (m < a.n) {
            a.ub_out[3 * m] = a.ubm[3 * m] + a.dt_rho * acc0;
            a.ub_out[3 * m + 1] = a.ubm[3 * m + 1] + a.dt_rho * acc1;
            a.ub_out[3 * m + 2] = a.ubm[3 * m + 2] + a.dt_rho * acc2;
            a.vb_out[3 * m] = a.damp * wm0;
            a.vb_out[3 * m + 1] = a.damp * wm1;
            a.vb_out[3 * m + 2] = a.damp * wm2;
            const uint32_t cls = a.bcc[m];
            if (cls) {
                const BcClass& bc = a.bct[cls];
                a.gl[m] += bc.force[0] * wm0 + bc.force[1] * wm1 + bc.force[2] * wm2;
            }
        }
    }
}

// u of every node (library order) from the FP64 records
__global__ void k_extract_u(const double* __restrict__ rec, int64_t n, double* __restrict__ u)
{
    GRID_STRIDE(e, 3 * n)
    {
        const int64_t p = e / 3;
        u[e] = rec[8 * p + 4 + (e - 3 * p)];
    }
}

// u of every node into the FP64 records (positions untouched)
__global__ void k_insert_u(const double* __restrict__ u, int64_t n, double* __restrict__ rec)
{
    GRID_STRIDE(e, 3 * n)
    {
        const int64_t p = e / 3;
        rec[8 * p + 4 + (e - 3 * p)] = u[e];
    }
}

// caller order <-> library order for 3-vectors per node
__global__ void k_to_lib3(const double* __restrict__ in, const int32_t* __restrict__ gid, int64_t n,
                          double* __restrict__ out)
{
    GRID_STRIDE(e, 3 * n)
    {
        const int64_t p = e / 3;
        out[e] = in[3 * (int64_t)gid[p] + (e - 3 * p)];
    }
}

__global__ void k_from_lib3(const double* __restrict__ in, const int32_t* __restrict__ gid,
                            int64_t n, double* __restrict__ out)
{
    GRID_STRIDE(e, 3 * n)
    {
        const int64_t p = e / 3;
        out[3 * (int64_t)gid[p] + (e - 3 * p)] = in[e];
    }
}

// Deterministic sum: each block reduces a contiguous chunk (fixed tree order)
// into partial[b]; one block then reduces the partials.
constexpr int kRedBlock = 256;

__device__ double block_sum(double v)
{
    __shared__ double sh[kRedBlock];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kRedBlock / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    return sh[0];
}

__global__ void __launch_bounds__(kRedBlock) k_sum_partial(const double* __restrict__ x, int64_t n,
                                                           int64_t chunk, double* __restrict__ partial)
{
    const int64_t lo = blockIdx.x * chunk;
    const int64_t hi = min(n, lo + chunk);
    double acc = 0.0;
    for (int64_t k = lo + threadIdx.x; k < hi; k += kRedBlock) acc += x[k];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kRedBlock) k_sum_final(const double* __restrict__ partial,
                                                         int nb, double scale,
                                                         double* __restrict__ out)
{
    double acc = 0.0;
    for (int k = threadIdx.x; k < nb; k += kRedBlock) acc += partial[k];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) *out = scale * s;
}

// canonical position of each used SELL slot of library node p: row gid[p] of
// the canonical family (sorted ids), found by binary search for the caller id
// of the slot's neighbour; out[position] = slot value
__global__ void k_slots_to_canonical(const double* __restrict__ val, const int32_t* __restrict__ nbr,
                                     const int32_t* __restrict__ gid, const int64_t* __restrict__ off,
                                     const int32_t* __restrict__ idx, int64_t n, int Q,
                                     double* __restrict__ out)
{
    const int64_t W = 32LL * Q;
    GRID_STRIDE(p, n)
    {
        const int64_t g = p >> 5, l = p & 31;
        const int64_t i = gid[p];
        const int64_t b = off[i], cnt = off[i + 1] - b;
        for (int64_t m = 0; m < cnt; ++m) {
            const int64_t slot = (g * W + m) * 32 + l;
            const int32_t j = gid[nbr[slot]];
            int64_t lo = 0, hi = cnt;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (idx[b + mid] < j) lo = mid + 1;
                else hi = mid;
            }
            if (lo < cnt) out[b + lo] = val[slot];
        }
    }
}

}  // namespace

cudaError_t launch_adj_mask(const double* ub, const double* vb, const uint8_t* bcc,
                            const BcClass* bct, int64_t n, double dt, double ws, double* ubm,
                            double* w, cudaStream_t s)
{
    k_adj_mask<<<grid_for(n, 256), 256, 0, s>>>(ub, vb, bcc, bct, n, dt, ws, ubm, w);
    return cudaGetLastError();
}

cudaError_t launch_adj_step(const AdjArgs& a, int grid, int block, cudaStream_t s)
{
    k_adj_step<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_extract_u(const double* rec, int64_t n, double* u, cudaStream_t s)
{
    k_extract_u<<<grid_for(3 * n, 256), 256, 0, s>>>(rec, n, u);
    return cudaGetLastError();
}

cudaError_t launch_insert_u(const double* u, int64_t n, double* rec, cudaStream_t s)
{
    k_insert_u<<<grid_for(3 * n, 256), 256, 0, s>>>(u, n, rec);
    return cudaGetLastError();
}

cudaError_t launch_to_lib3(const double* in, const int32_t* gid, int64_t n, double* out,
                           cudaStream_t s)
{
    k_to_lib3<<<grid_for(3 * n, 256), 256, 0, s>>>(in, gid, n, out);
    return cudaGetLastError();
}

cudaError_t launch_from_lib3(const double* in, const int32_t* gid, int64_t n, double* out,
                             cudaStream_t s)
{
    k_from_lib3<<<grid_for(3 * n, 256), 256, 0, s>>>(in, gid, n, out);
    return cudaGetLastError();
}

int sum_partials_needed(int64_t n) { return (int)std::min<int64_t>(1024, (n + 4095) / 4096 + 1); }

cudaError_t launch_sum(const double* x, int64_t n, double scale, double* partial, int n_partial,
                       double* out, cudaStream_t s)
{
    const int64_t chunk = (n + n_partial - 1) / n_partial;
    k_sum_partial<<<n_partial, kRedBlock, 0, s>>>(x, n, chunk > 0 ? chunk : 1, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_final<<<1, kRedBlock, 0, s>>>(partial, n_partial, scale, out);
    return cudaGetLastError();
}

cudaError_t launch_slots_to_canonical(const double* val, const int32_t* nbr, const int32_t* gid,
                                      const int64_t* off, const int32_t* idx, int64_t n, int Q,
                                      double* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_slots_to_canonical<<<grid_for(n, 128), 128, 0, s>>>(val, nbr, gid, off, idx, n, Q, out);
    return cudaGetLastError();
}

}  // namespace pd
