// Auxiliary kernels: step counter, state transfer between the caller's node
// order and the library's spatial order, damage from the bond flags (Eq. 8),
// and the per-node bond weights w = c V.
#include <cuda_runtime.h>

#include "pd_internal.h"

namespace pd {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__global__ void k_advance(int64_t* ctr, int64_t k)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *ctr += k;
}

__global__ void k_get_state_f32(const double* __restrict__ u64, const float* __restrict__ v32,
                                const int32_t* __restrict__ gid, int64_t n,
                                double* __restrict__ u_out, double* __restrict__ v_out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / 3;
        const int c = (int)(e - 3 * p);
        const int64_t g = gid[p];
        if (u_out) u_out[3 * g + c] = u64[e];
        if (v_out) v_out[3 * g + c] = (double)v32[e];
    }
}

__global__ void k_set_state_f32(const double* __restrict__ u_in, const double* __restrict__ v_in,
                                const int32_t* __restrict__ gid, int64_t n, double inv_delta,
                                double* __restrict__ u64, float4* __restrict__ rec,
                                float* __restrict__ v32)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = gid[p];
        if (u_in) {
            const double ux = u_in[3 * g], uy = u_in[3 * g + 1], uz = u_in[3 * g + 2];
            u64[3 * p] = ux;
            u64[3 * p + 1] = uy;
            u64[3 * p + 2] = uz;
            rec[2 * p + 1] = make_float4((float)(ux * inv_delta), (float)(uy * inv_delta),
                                         (float)(uz * inv_delta), 0.0f);
        }
        if (v_in) {
            for (int c = 0; c < 3; ++c) v32[3 * p + c] = (float)v_in[3 * g + c];
        }
    }
}

__global__ void k_get_state_f64(const double* __restrict__ rec, const double* __restrict__ v64,
                                const int32_t* __restrict__ gid, int64_t n,
                                double* __restrict__ u_out, double* __restrict__ v_out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / 3;
        const int c = (int)(e - 3 * p);
        const int64_t g = gid[p];
        if (u_out) u_out[3 * g + c] = rec[8 * p + 4 + c];
        if (v_out) v_out[3 * g + c] = v64[e];
    }
}

__global__ void k_set_state_f64(const double* __restrict__ u_in, const double* __restrict__ v_in,
                                const int32_t* __restrict__ gid, int64_t n,
                                double* __restrict__ rec, double* __restrict__ v64)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 3 * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / 3;
        const int c = (int)(e - 3 * p);
        const int64_t g = gid[p];
        if (u_in) rec[8 * p + 4 + c] = u_in[3 * g + c];
        if (v_in) v64[e] = v_in[3 * g + c];
    }
}

template <typename T>
__device__ __forceinline__ T rec_w(const void* rec, int64_t p);
template <>
__device__ __forceinline__ float rec_w<float>(const void* rec, int64_t p)
{
    return reinterpret_cast<const float4*>(rec)[2 * p].w;
}
template <>
__device__ __forceinline__ double rec_w<double>(const void* rec, int64_t p)
{
    return reinterpret_cast<const double*>(rec)[8 * p + 3];
}

// phi = 1 - sum_{intact j} w_j / sum_{family j} w_j  (Eq. 8), warp per node.
template <typename T>
__global__ void k_damage(const void* __restrict__ rec, const int32_t* __restrict__ nbr,
                         const uint32_t* __restrict__ bits, const T* __restrict__ wsum_inv,
                         const int32_t* __restrict__ gid, int64_t n, int Q,
                         double* __restrict__ phi)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += nw) {
        T acc = 0;
        for (int q = 0; q < Q; ++q) {
            const uint32_t w = bits[p * Q + q];
            if ((w >> lane) & 1u) acc += rec_w<T>(rec, nbr[p * 32 * Q + q * 32 + lane]);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) phi[gid[p]] = (double)(1 - acc * wsum_inv[p]);
    }
}

template <typename T>
__global__ void k_set_w(void* rec0, void* rec1, const double* __restrict__ vol, int64_t n,
                        double wscale)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const T w = (T)(wscale * vol[p]);
        if (sizeof(T) == 4) {
            reinterpret_cast<float4*>(rec0)[2 * p].w = (float)w;
            reinterpret_cast<float4*>(rec1)[2 * p].w = (float)w;
        } else {
            reinterpret_cast<double*>(rec0)[8 * p + 3] = (double)w;
            reinterpret_cast<double*>(rec1)[8 * p + 3] = (double)w;
        }
    }
}

template <typename T>
__global__ void k_wsum(const void* __restrict__ rec, const int32_t* __restrict__ nbr,
                       const int32_t* __restrict__ fam_cnt, int64_t n, int Q,
                       T* __restrict__ wsum_inv)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < n; p += nw) {
        T acc = 0;
        const int cnt = fam_cnt[p];
        for (int q = 0; q < Q; ++q) {
            const int m = q * 32 + lane;
            if (m < cnt) acc += rec_w<T>(rec, nbr[p * 32 * Q + m]);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (lane == 0) wsum_inv[p] = acc > 0 ? (T)1 / acc : (T)0;
    }
}

template <typename T>
__global__ void k_gather_damage(const T* __restrict__ dmg, const int32_t* __restrict__ gid,
                                int64_t n, double* __restrict__ phi)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x)
        phi[gid[p]] = (double)dmg[p];
}

int grid_for(int64_t work, int block)
{
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 65535 * 8) g = 65535 * 8;
    return (int)g;
}

}  // namespace

cudaError_t launch_advance(int64_t* step_ctr, int64_t k, cudaStream_t s)
{
    k_advance<<<1, 32, 0, s>>>(step_ctr, k);
    return cudaGetLastError();
}

cudaError_t launch_get_state_f32(const double* u64, const float* v32, const int32_t* gid,
                                 int64_t n, double* u_out, double* v_out, cudaStream_t s)
{
    k_get_state_f32<<<grid_for(3 * n, 256), 256, 0, s>>>(u64, v32, gid, n, u_out, v_out);
    return cudaGetLastError();
}

cudaError_t launch_set_state_f32(const double* u_in, const double* v_in, const int32_t* gid,
                                 int64_t n, double inv_delta, double* u64, float4* rec,
                                 float* v32, cudaStream_t s)
{
    k_set_state_f32<<<grid_for(n, 256), 256, 0, s>>>(u_in, v_in, gid, n, inv_delta, u64, rec,
                                                     v32);
    return cudaGetLastError();
}

cudaError_t launch_get_state_f64(const double* rec64, const double* v64, const int32_t* gid,
                                 int64_t n, double* u_out, double* v_out, cudaStream_t s)
{
    k_get_state_f64<<<grid_for(3 * n, 256), 256, 0, s>>>(rec64, v64, gid, n, u_out, v_out);
    return cudaGetLastError();
}

cudaError_t launch_set_state_f64(const double* u_in, const double* v_in, const int32_t* gid,
                                 int64_t n, double* rec64, double* v64, cudaStream_t s)
{
    k_set_state_f64<<<grid_for(3 * n, 256), 256, 0, s>>>(u_in, v_in, gid, n, rec64, v64);
    return cudaGetLastError();
}

cudaError_t launch_damage(int precision, const void* rec, const int32_t* nbr,
                          const uint32_t* bits, const void* wsum_inv, const int32_t* gid,
                          int64_t n, int Q, double* phi_out, cudaStream_t s)
{
    const int g = grid_for(32 * n, 256);
    if (precision == 32)
        k_damage<float><<<g, 256, 0, s>>>(rec, nbr, bits, (const float*)wsum_inv, gid, n, Q,
                                          phi_out);
    else
        k_damage<double><<<g, 256, 0, s>>>(rec, nbr, bits, (const double*)wsum_inv, gid, n, Q,
                                           phi_out);
    return cudaGetLastError();
}

cudaError_t launch_gather_damage(int precision, const void* dmg, const int32_t* gid, int64_t n,
                                 double* phi_out, cudaStream_t s)
{
    if (precision == 32)
        k_gather_damage<float><<<grid_for(n, 256), 256, 0, s>>>((const float*)dmg, gid, n, phi_out);
    else
        k_gather_damage<double><<<grid_for(n, 256), 256, 0, s>>>((const double*)dmg, gid, n,
                                                                 phi_out);
    return cudaGetLastError();
}

cudaError_t launch_set_weights(int precision, void* rec0, void* rec1, const double* vol,
                               const int32_t* nbr, const int32_t* fam_cnt, int64_t n, int Q,
                               double wscale, void* wsum_inv, cudaStream_t s)
{
    if (precision == 32) {
        k_set_w<float><<<grid_for(n, 256), 256, 0, s>>>(rec0, rec1, vol, n, wscale);
        k_wsum<float><<<grid_for(32 * n, 256), 256, 0, s>>>(rec0, nbr, fam_cnt, n, Q,
                                                            (float*)wsum_inv);
    } else {
        k_set_w<double><<<grid_for(n, 256), 256, 0, s>>>(rec0, rec1, vol, n, wscale);
        k_wsum<double><<<grid_for(32 * n, 256), 256, 0, s>>>(rec0, nbr, fam_cnt, n, Q,
                                                             (double*)wsum_inv);
    }
    return cudaGetLastError();
}

}  // namespace pd
