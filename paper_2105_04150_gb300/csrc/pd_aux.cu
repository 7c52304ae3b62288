// Auxiliary kernels: step counter, state transfer between the caller's node
// order and the library's node order, damage from the bond flags (Eq. 8),
// and the per-node bond weights w = c V.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pd_internal.h"

namespace pd {
namespace {

__global__ void k_advance(int64_t* ctr, int64_t k)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *ctr += k;
}

#define GRID_STRIDE(var, count)                                                   \
    for (int64_t var = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; var < (count); \
         var += (int64_t)gridDim.x * blockDim.x)

__global__ void k_get_state_f32(const float4* __restrict__ rec, const float4* __restrict__ lo32,
                                const float* __restrict__ v32, const int32_t* __restrict__ gid,
                                int64_t n, double delta, double* __restrict__ u_out,
                                double* __restrict__ v_out)
{
    GRID_STRIDE(p, n)
    {
        const int64_t g = gid[p];
        if (u_out) {
            const float4 a = rec[2 * p], b = rec[2 * p + 1], l = lo32[p];
            u_out[3 * g] = ((double)a.w + (double)l.x) * delta;
            u_out[3 * g + 1] = ((double)b.x + (double)l.y) * delta;
            u_out[3 * g + 2] = ((double)b.y + (double)l.z) * delta;
        }
        if (v_out)
            for (int c = 0; c < 3; ++c) v_out[3 * g + c] = (double)v32[3 * p + c];
    }
}

__device__ __forceinline__ void split(double x, float& h, float& l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

__device__ __forceinline__ float bf16_pair(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return __uint_as_float(*reinterpret_cast<const uint32_t*>(&v));
}

__global__ void k_set_state_f32(const double* __restrict__ u_in, const double* __restrict__ v_in,
                                const int32_t* __restrict__ gid, int64_t n, double inv_delta,
                                float4* __restrict__ rec, float4* __restrict__ lo32,
                                float* __restrict__ v32)
{
    GRID_STRIDE(p, n)
    {
        const int64_t g = gid[p];
        if (u_in) {
            float h[3], l[3];
            for (int c = 0; c < 3; ++c) split(u_in[3 * g + c] * inv_delta, h[c], l[c]);
            float4 a = rec[2 * p];
            a.w = h[0];
            rec[2 * p] = a;
            // same packing as the step kernel: {bf16(l_x) | bf16(l_y)}, {bf16(l_z) | 0}
            rec[2 * p + 1] = make_float4(h[1], h[2], bf16_pair(l[1], l[0]), bf16_pair(0.0f, l[2]));
            lo32[p] = make_float4(l[0], l[1], l[2], 0.0f);
        }
        if (v_in)
            for (int c = 0; c < 3; ++c) v32[3 * p + c] = (float)v_in[3 * g + c];
    }
}

__global__ void k_get_state_lat(const double* __restrict__ ul, const float* __restrict__ v32,
                                const int32_t* __restrict__ gid, int64_t n, double delta,
                                const int32_t* __restrict__ inst,
                                const InstParams* __restrict__ itab, double* __restrict__ u_out,
                                double* __restrict__ v_out)
{
    GRID_STRIDE(e, 3 * n)
    {
        const int64_t p = e / 3;
        const int c = (int)(e - 3 * p);
        const int64_t g = gid[p];
        const double unit = inst ? itab[inst[p]].unit : delta;
        if (u_out) u_out[3 * g + c] = ul[e] * unit;
        if (v_out) v_out[3 * g + c] = (double)v32[e];
    }
}

__global__ void k_set_state_lat(const double* __restrict__ u_in, const double* __restrict__ v_in,
                                const int32_t* __restrict__ gid, int64_t n, double inv_delta,
                                const int32_t* __restrict__ inst,
                                const InstParams* __restrict__ itab, double* __restrict__ ul,
                                float4* __restrict__ pub, float* __restrict__ v32)
{
    GRID_STRIDE(p, n)
    {
        const int64_t g = gid[p];
        if (u_in) {
            const double inv_unit = inst ? itab[inst[p]].inv_unit : inv_delta;
            double u[3];
            for (int c = 0; c < 3; ++c) {
                u[c] = u_in[3 * g + c] * inv_unit;
                ul[3 * p + c] = u[c];
            }
            pub[p] = make_float4((float)u[0], (float)u[1], (float)u[2], 0.0f);
        }
        if (v_in)
            for (int c = 0; c < 3; ++c) v32[3 * p + c] = (float)v_in[3 * g + c];
    }
}

__global__ void k_get_state_f64(const double* __restrict__ rec, const double* __restrict__ v64,
                                const int32_t* __restrict__ gid, int64_t n,
                                double* __restrict__ u_out, double* __restrict__ v_out)
{
    GRID_STRIDE(e, 3 * n)
    {
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
    GRID_STRIDE(e, 3 * n)
    {
        const int64_t p = e / 3;
        const int c = (int)(e - 3 * p);
        const int64_t g = gid[p];
        if (u_in) rec[8 * p + 4 + c] = u_in[3 * g + c];
        if (v_in) v64[e] = v_in[3 * g + c];
    }
}

template <typename T>
__device__ __forceinline__ T node_w(const void* wrec, int64_t p);
template <>
__device__ __forceinline__ float node_w<float>(const void* wrec, int64_t p)
{
    return reinterpret_cast<const float*>(wrec)[p];
}
template <>
__device__ __forceinline__ double node_w<double>(const void* wrec, int64_t p)
{
    return reinterpret_cast<const double*>(wrec)[8 * p + 3];
}

// sum over the set bits of `bits` of w_j, lane per node, in slot order (the
// same order as the step kernels, so the result is bit-identical to theirs).
template <typename T>
__device__ __forceinline__ T masked_wsum(const void* wrec, const int32_t* __restrict__ nbr,
                                         const uint32_t* __restrict__ bits, int64_t g, int lane,
                                         int Wg, int Q, const T* __restrict__ integ = nullptr)
{
    const int64_t W = 32LL * Q;
    T acc = 0;
    for (int q = 0; q * 32 < Wg; ++q) {
        const uint32_t word = bits[(g * Q + q) * 32 + lane];
        const int mend = min(32, Wg - q * 32);
        for (int b = 0; b < mend; ++b)
            if ((word >> b) & 1u) {
                const int64_t slot = (g * W + q * 32 + b) * 32 + lane;
                const T w = node_w<T>(wrec, nbr[slot]);
                acc += integ != nullptr ? w * integ[slot] : w;
            }
    }
    return acc;
}

template <typename T>
__global__ void k_damage(const void* __restrict__ wrec, const int32_t* __restrict__ nbr,
                         const uint32_t* __restrict__ bits, const int32_t* __restrict__ sw,
                         const T* __restrict__ wsum_inv, const int32_t* __restrict__ gid,
                         int64_t n, int Q, const T* __restrict__ integ, double* __restrict__ phi)
{
    GRID_STRIDE(p, ((n + 31) >> 5) << 5)
    {
        const int64_t g = p >> 5;
        const int lane = (int)(p & 31);
        const T acc = masked_wsum<T>(wrec, nbr, bits, g, lane, sw[g], Q, integ);
        // a node without family has no damage (the integral ratio of Eq. 8 is 0/0)
        if (p < n)
            phi[gid[p]] = wsum_inv[p] > 0 ? (double)fmax((T)0, (T)1 - acc * wsum_inv[p]) : 0.0;
    }
}

template <typename T>
__global__ void k_gather_damage(const T* __restrict__ dmg, const int32_t* __restrict__ gid,
                                int64_t n, double* __restrict__ phi)
{
    GRID_STRIDE(p, n) phi[gid[p]] = (double)dmg[p];
}

template <typename T>
__global__ void k_set_w(void* wrec0, void* wrec1, const double* __restrict__ vol, int64_t n,
                        double wscale)
{
    GRID_STRIDE(p, n)
    {
        if (sizeof(T) == 4) {
            reinterpret_cast<float*>(wrec0)[p] = (float)(wscale * vol[p]);
        } else {
            reinterpret_cast<double*>(wrec0)[8 * p + 3] = wscale * vol[p];
            reinterpret_cast<double*>(wrec1)[8 * p + 3] = wscale * vol[p];
        }
    }
}

template <typename T>
__global__ void k_wsum(const void* __restrict__ wrec, const int32_t* __restrict__ nbr,
                       const uint32_t* __restrict__ bits0, const int32_t* __restrict__ sw,
                       int64_t n, int Q, T* __restrict__ wsum_inv)
{
    GRID_STRIDE(p, ((n + 31) >> 5) << 5)
    {
        const int64_t g = p >> 5;
        const int lane = (int)(p & 31);
        const T acc = masked_wsum<T>(wrec, nbr, bits0, g, lane, sw[g], Q);
        wsum_inv[p] = acc > 0 ? (T)1 / acc : (T)0;
    }
}

__global__ void k_inv_len(const double* __restrict__ x64, const int32_t* __restrict__ nbr,
                          const int32_t* __restrict__ sw, int64_t n, int Q,
                          double* __restrict__ ilen)
{
    const int64_t W = 32LL * Q;
    GRID_STRIDE(p, ((n + 31) >> 5) << 5)
    {
        const int64_t g = p >> 5;
        const int lane = (int)(p & 31);
        const int Wg = sw[g];
        for (int m = 0; m < Wg; ++m) {
            const int64_t slot = (g * W + m) * 32 + lane;
            const int64_t j = nbr[slot];
            double v = 0.0;
            if (j != p) {
                const double ex = x64[3 * j] - x64[3 * p], ey = x64[3 * j + 1] - x64[3 * p + 1],
                             ez = x64[3 * j + 2] - x64[3 * p + 2];
                v = 1.0 / sqrt(ex * ex + ey * ey + ez * ez);
            }
            ilen[slot] = v;
        }
    }
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

cudaError_t launch_get_state_f32(const float4* rec, const float4* lo32, const float* v32,
                                 const int32_t* gid, int64_t n, double delta, double* u_out,
                                 double* v_out, cudaStream_t s)
{
    k_get_state_f32<<<grid_for(n, 256), 256, 0, s>>>(rec, lo32, v32, gid, n, delta, u_out,
                                                     v_out);
    return cudaGetLastError();
}

cudaError_t launch_set_state_f32(const double* u_in, const double* v_in, const int32_t* gid,
                                 int64_t n, double inv_delta, float4* rec, float4* lo32,
                                 float* v32, cudaStream_t s)
{
    k_set_state_f32<<<grid_for(n, 256), 256, 0, s>>>(u_in, v_in, gid, n, inv_delta, rec, lo32,
                                                     v32);
    return cudaGetLastError();
}

cudaError_t launch_get_state_lat(const double* u_lat, const float* v32, const int32_t* gid,
                                 int64_t n, double delta, const int32_t* inst,
                                 const InstParams* itab, double* u_out, double* v_out,
                                 cudaStream_t s)
{
    k_get_state_lat<<<grid_for(3 * n, 256), 256, 0, s>>>(u_lat, v32, gid, n, delta, inst, itab,
                                                         u_out, v_out);
    return cudaGetLastError();
}

cudaError_t launch_set_state_lat(const double* u_in, const double* v_in, const int32_t* gid,
                                 int64_t n, double inv_delta, const int32_t* inst,
                                 const InstParams* itab, double* u_lat, float4* pub, float* v32,
                                 cudaStream_t s)
{
    k_set_state_lat<<<grid_for(n, 256), 256, 0, s>>>(u_in, v_in, gid, n, inv_delta, inst, itab,
                                                     u_lat, pub, v32);
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

cudaError_t launch_damage(int precision, const void* wrec, const int32_t* nbr,
                          const uint32_t* bits, const int32_t* sw, const void* wsum_inv,
                          const int32_t* gid, int64_t n, int Q, const void* integ,
                          double* phi_out, cudaStream_t s)
{
    const int g = grid_for(n, 256);
    if (precision == 32)
        k_damage<float><<<g, 256, 0, s>>>(wrec, nbr, bits, sw, (const float*)wsum_inv, gid, n, Q,
                                          (const float*)integ, phi_out);
    else
        k_damage<double><<<g, 256, 0, s>>>(wrec, nbr, bits, sw, (const double*)wsum_inv, gid, n,
                                           Q, (const double*)integ, phi_out);
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

cudaError_t launch_set_weights(int precision, void* wrec0, void* wrec1, const double* vol,
                               const int32_t* nbr, const uint32_t* init_bits, const int32_t* sw,
                               int64_t n, int Q, double wscale, void* wsum_inv, cudaStream_t s)
{
    if (precision == 32) {
        k_set_w<float><<<grid_for(n, 256), 256, 0, s>>>(wrec0, wrec1, vol, n, wscale);
        k_wsum<float><<<grid_for(n, 256), 256, 0, s>>>(wrec0, nbr, init_bits, sw, n, Q,
                                                       (float*)wsum_inv);
    } else {
        k_set_w<double><<<grid_for(n, 256), 256, 0, s>>>(wrec0, wrec1, vol, n, wscale);
        k_wsum<double><<<grid_for(n, 256), 256, 0, s>>>(wrec0, nbr, init_bits, sw, n, Q,
                                                        (double*)wsum_inv);
    }
    return cudaGetLastError();
}

__global__ void k_check_finite(const double* __restrict__ x, int64_t m, int* __restrict__ flag)
{
    bool bad = false;
    GRID_STRIDE(e, m) bad = bad || !isfinite(x[e]);
    if (bad) atomicOr(flag, 1);
}

template <typename T>
__global__ void k_fill(T* __restrict__ dst, int64_t n, T v)
{
    GRID_STRIDE(e, n) dst[e] = v;
}

// clear bond-flag bits (word index, mask of bits to clear) and zero the
// integrity of the same slots (softening handles)
__global__ void k_clear_slots(uint32_t* __restrict__ bits, const int64_t* __restrict__ word,
                              const uint32_t* __restrict__ mask, const int64_t* __restrict__ slot,
                              int64_t m, int precision, void* integ)
{
    GRID_STRIDE(e, m)
    {
        atomicAnd(bits + word[e], ~mask[e]);
        if (integ != nullptr) {
            if (precision == 32)
                static_cast<float*>(integ)[slot[e]] = 0.0f;
            else
                static_cast<double*>(integ)[slot[e]] = 0.0;
        }
    }
}

cudaError_t launch_clear_slots(uint32_t* bits, const int64_t* word, const uint32_t* mask,
                               const int64_t* slot, int64_t m, int precision, void* integ,
                               cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_clear_slots<<<grid_for(m, 256), 256, 0, s>>>(bits, word, mask, slot, m, precision, integ);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const double* x, int64_t m, int* flag, cudaStream_t s)
{
    if (m <= 0) return cudaSuccess;
    k_check_finite<<<grid_for(m, 256), 256, 0, s>>>(x, m, flag);
    return cudaGetLastError();
}

cudaError_t launch_fill(int precision, void* dst, int64_t n, double v, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (precision == 32)
        k_fill<float><<<grid_for(n, 256), 256, 0, s>>>((float*)dst, n, (float)v);
    else
        k_fill<double><<<grid_for(n, 256), 256, 0, s>>>((double*)dst, n, v);
    return cudaGetLastError();
}

cudaError_t launch_inv_len(const double* x64, const int32_t* nbr, const int32_t* sw, int64_t n,
                           int Q, double* ilen, cudaStream_t s)
{
    k_inv_len<<<grid_for(((n + 31) >> 5) << 5, 256), 256, 0, s>>>(x64, nbr, sw, n, Q, ilen);
    return cudaGetLastError();
}

}  // namespace pd
