// Fused FP64 peridynamic step kernel for sm_103a (the parity path).
//
// Same decomposition as the FP32-bulk kernel (warp per 32-node group, lane
// per family member, shuffle reduction, lane-parallel integration, bit-packed
// bond flags, double-buffered node records), but every quantity is FP64 and
// the stretch is the literal one of Eq. 4, s = (|xi+eta| - |xi|) / |xi|, so
// the break decisions are FP64 decisions.  Node record: 8 doubles
// {x, y, z, w, ux, uy, uz, 0} with w = c V_j (or V_j with per-bond c).
#include <cuda_runtime.h>

#include "pd_internal.h"

namespace pd {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t splitmix_out(uint64_t seed, uint64_t m)
{
    uint64_t z = seed + m * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double sc_draw(uint64_t seed, double lo, double hi, int32_t gi,
                                          int32_t gj)
{
    const uint64_t a = (uint64_t)(uint32_t)min(gi, gj);
    const uint64_t b = (uint64_t)(uint32_t)max(gi, gj);
    const uint64_t h = splitmix_out(seed, ((a << 32) | b) + 1ull);
    return lo + (hi - lo) * ((double)(h >> 11) * 0x1.0p-53);
}

__device__ __noinline__ bool pair_no_fail(const uint8_t* __restrict__ bcc,
                                          const BcClass* __restrict__ bct, int64_t i, int64_t j)
{
    return ((bct[bcc[i]].mask | bct[bcc[j]].mask) & 8u) != 0u;
}

template <int QT, int SCM>
__global__ void __launch_bounds__(256) k_step_f64(const StepArgsF64 a)
{
    const int Q = (QT > 0) ? QT : a.q_rt;
    const int W = 32 * Q;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = *a.step_ctr + a.k;
    const int cur = (int)(step & 1);
    const double2* __restrict__ rin = reinterpret_cast<const double2*>(a.rec[cur]);
    double2* __restrict__ rout = reinterpret_cast<double2*>(const_cast<double*>(a.rec[cur ^ 1]));
    const double* __restrict__ cb = a.cbond;
    const int64_t ngroups = (a.n + 31) >> 5;

    for (int64_t g = wid; g < ngroups; g += nwarps) {
        const int64_t base = g << 5;
        const int cnt = (int)min((int64_t)32, a.n - base);
        double kx = 0.0, ky = 0.0, kz = 0.0, kw = 0.0;

        for (int t = 0; t < cnt; ++t) {
            const int64_t i = base + t;
            const double2 x01 = __ldg(rin + 4 * i), x23 = __ldg(rin + 4 * i + 1);
            const double2 u01 = __ldg(rin + 4 * i + 2), u23 = __ldg(rin + 4 * i + 3);
            const int32_t* __restrict__ row = a.nbr + i * W;
            uint32_t* brow = a.bits + i * Q;
            double fx = 0.0, fy = 0.0, fz = 0.0, ws = 0.0;

            for (int q0 = 0; q0 < Q; q0 += 2) {
                uint32_t w[2];
                int32_t jj[2];
                bool al[2];
                double2 ra[2][4];
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int q = q0 + c;
                    al[c] = false;
                    w[c] = 0u;
                    jj[c] = 0;
                    if (q < Q) {
                        w[c] = brow[q];
                        jj[c] = __ldg(row + q * 32 + lane);
                        al[c] = (w[c] >> lane) & 1u;
                    }
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (al[c]) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) ra[c][e] = __ldg(rin + 4 * (int64_t)jj[c] + e);
                    }
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (al[c]) {
                        const double ex = ra[c][0].x - x01.x, ey = ra[c][0].y - x01.y;
                        const double ez = ra[c][1].x - x23.x;
                        const double yx = ex + (ra[c][2].x - u01.x);
                        const double yy = ey + (ra[c][2].y - u01.y);
                        const double yz = ez + (ra[c][3].x - u23.x);
                        const double L = sqrt(ex * ex + ey * ey + ez * ez);
                        const double r = sqrt(yx * yx + yy * yy + yz * yz);
                        const double s = (r - L) / L;
                        const double sc = (SCM == 0)
                                              ? a.sc
                                              : sc_draw(a.sc_seed, a.sc_lo, a.sc_hi, a.gid[i],
                                                        a.gid[jj[c]]);
                        bool brk = s >= sc;
                        if (brk && a.has_nofail) brk = !pair_no_fail(a.bcc, a.bct, i, jj[c]);
                        if (brk) {
                            al[c] = false;
                        } else {
                            double wj = ra[c][1].y;
                            if (cb != nullptr) wj *= __ldg(cb + i * W + (q0 + c) * 32 + lane);
                            const double f = wj * s / r;
                            fx += f * yx;
                            fy += f * yy;
                            fz += f * yz;
                            ws += ra[c][1].y;
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (q0 + c < Q) {
                        const uint32_t nw = __ballot_sync(kFull, al[c]);
                        if (lane == 0 && nw != w[c]) brow[q0 + c] = nw;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                fx += __shfl_xor_sync(kFull, fx, o);
                fy += __shfl_xor_sync(kFull, fy, o);
                fz += __shfl_xor_sync(kFull, fz, o);
                ws += __shfl_xor_sync(kFull, ws, o);
            }
            if (lane == t) {
                kx = fx;
                ky = fy;
                kz = fz;
                kw = ws;
            }
        }

        if (lane < cnt) {
            const int64_t i = base + lane;
            const uint32_t cls = a.bcc[i];
            uint32_t mask = 0u;
            double gdisp[3] = {0.0, 0.0, 0.0};
            double F[3] = {kx, ky, kz};
            if (cls != 0u) {
                const BcClass& bc = a.bct[cls];
                mask = bc.mask;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    gdisp[c] = bc.disp[c];
                    F[c] += a.load * bc.force[c];
                }
            }
            const double s_now = a.disp_rate * (double)step;
            const double s_next = a.disp_rate * (double)(step + 1);
            const double2 r01 = __ldg(rin + 4 * i), r23 = __ldg(rin + 4 * i + 1);
            const double2 q01 = __ldg(rin + 4 * i + 2), q23 = __ldg(rin + 4 * i + 3);
            const double uo[3] = {q01.x, q01.y, q23.x};
            double un[3];
            bool finite = true;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double vi = a.v[3 * i + c];
                double vn = vi + a.dt * (F[c] - a.eta * vi) / a.rho;
                double u = uo[c] + a.dt * vn;
                if (mask & (1u << c)) {
                    u = gdisp[c] * s_next;
                    vn = gdisp[c] * (s_next - s_now) / a.dt;
                }
                finite = finite && isfinite(u);
                un[c] = u;
                a.v[3 * i + c] = vn;
            }
            rout[4 * i] = r01;
            rout[4 * i + 1] = r23;
            rout[4 * i + 2] = make_double2(un[0], un[1]);
            rout[4 * i + 3] = make_double2(un[2], 0.0);
            a.damage[i] = 1.0 - kw * a.wsum_inv[i];
            if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
        }
    }
}

template <int QT>
cudaError_t launch_q(const StepArgsF64& a, int sc_mode, int grid, int block, cudaStream_t s)
{
    if (sc_mode == 0)
        k_step_f64<QT, 0><<<grid, block, 0, s>>>(a);
    else
        k_step_f64<QT, 1><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int QT>
const void* kernel_ptr(int sc_mode)
{
    return sc_mode == 0 ? (const void*)k_step_f64<QT, 0> : (const void*)k_step_f64<QT, 1>;
}

}  // namespace

cudaError_t launch_step_f64(const StepArgsF64& a, int Q, int sc_mode, int grid, int block,
                            cudaStream_t s)
{
    switch (Q) {
        case 4: return launch_q<4>(a, sc_mode, grid, block, s);
        default: return launch_q<0>(a, sc_mode, grid, block, s);
    }
}

const void* step_f64_kernel(int Q, int sc_mode)
{
    switch (Q) {
        case 4: return kernel_ptr<4>(sc_mode);
        default: return kernel_ptr<0>(sc_mode);
    }
}

}  // namespace pd
