// Ordinary state-based peridynamics (linear peridynamic solid, constant
// influence function) in FP64: the two loops per step of the paper's
// "State-based Peridynamics" section as two lane-per-node kernels over the same
// sliced family layout as the bond-based step.
//
//   k_osb_dilation  per node: bonds past s_c break (Eq. 6, s = e / |xi|), then
//                   theta_i = (3 / m_i) sum_j mu_ij |xi| e_ij V_j, e = |y| - |xi|
//   k_osb_force     per node: F_i = sum_j mu_ij (t_ij + t_ji) V_j y / |y| with
//                   t_ij = (3 K theta_i / m_i) |xi| + (15 G / m_i)(e - theta_i |xi| / 3);
//                   then the damped Euler-Cromer or velocity-Verlet update,
//                   boundary conditions and damage of the bond-based FP64 step
//
// m_i = sum_j |xi|^2 V_j over the family after the initial cuts, computed once.
// t_ij is linear in the bond: t_ij = alpha_i |xi| + beta_i e with
// beta_i = 15 G / m_i (once) and alpha_i = 3 K theta_i / m_i - beta_i theta_i / 3
// (written by the dilation kernel), so the force loop gathers two coefficients
// per neighbour and divides nothing (FP64 division is costly on GB300).
// The record layout, double buffering and step counter are the FP64 step's.
#include <cuda_runtime.h>

#include "pd_internal.h"

namespace pd {
namespace {

__device__ __forceinline__ uint64_t splitmix_out(uint64_t seed, uint64_t m)
{
    uint64_t z = seed + m * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double bond_sc(const StepArgsF64& a, int64_t i, int64_t j)
{
    double lo_sc = a.sc_lo, hi_sc = a.sc_hi, sc = a.sc;
    uint64_t seed = a.sc_seed, gi, gj;
    if (a.inst != nullptr) {  // batch: the instance's parameters, instance-local ids as keys
        const InstParams& ip = a.itab[a.inst[i]];
        if (ip.sc_mode == 0) return ip.sc;
        lo_sc = ip.sc_lo;
        hi_sc = ip.sc_hi;
        seed = ip.sc_seed;
        gi = (uint32_t)a.hid[i];
        gj = (uint32_t)a.hid[j];
    } else {
        if (lo_sc == hi_sc) return sc;
        gi = (uint32_t)a.gid[i];
        gj = (uint32_t)a.gid[j];
    }
    const uint64_t lo = gi < gj ? gi : gj, hi = gi < gj ? gj : gi;
    const uint64_t h = splitmix_out(seed, ((lo << 32) | hi) + 1ull);
    return lo_sc + (hi_sc - lo_sc) * ((double)(h >> 11) * 0x1.0p-53);
}

// deformed bond vector and its length from the records of i and j
struct OsbBond {
    double y0, y1, y2, r, ir;
};

__device__ __forceinline__ OsbBond osb_bond(const double2* __restrict__ rin, int64_t i, int64_t j)
{
    const double2 xi01 = rin[4 * i], xi23 = rin[4 * i + 1], ui01 = rin[4 * i + 2],
                  ui23 = rin[4 * i + 3];
    const double2 xj01 = __ldg(rin + 4 * j), xj23 = __ldg(rin + 4 * j + 1),
                  uj01 = __ldg(rin + 4 * j + 2), uj23 = __ldg(rin + 4 * j + 3);
    OsbBond b;
    b.y0 = (xj01.x - xi01.x) + (uj01.x - ui01.x);
    b.y1 = (xj01.y - xi01.y) + (uj01.y - ui01.y);
    b.y2 = (xj23.x - xi23.x) + (uj23.x - ui23.x);
    const double q = b.y0 * b.y0 + b.y1 * b.y1 + b.y2 * b.y2;
    b.ir = rsqrt_nr(q);
    b.r = q * b.ir;
    return b;
}

__global__ void __launch_bounds__(256) k_osb_weighted_volume(const StepArgsF64 a, OsbArgs o)
{
    const int64_t W = 32LL * a.Q;
    const int64_t nslices = (a.n + 31) >> 5;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nslices * 32;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = p >> 5;
        const int lane = (int)(p & 31);
        double acc = 0.0;
        for (int q = 0; q * 32 < a.sw[g]; ++q) {
            const uint32_t word = a.bits[(g * a.Q + q) * 32 + lane];
            for (int b = 0; b < 32 && q * 32 + b < a.sw[g]; ++b) {
                if (!((word >> b) & 1u)) continue;
                const int64_t slot = (g * W + q * 32 + b) * 32 + lane;
                const double L = o.len[slot];
                acc += L * L * o.vol[a.nbr[slot]];
            }
        }
        o.mvol[p] = acc;
        o.beta[p] = acc > 0.0 ? 15.0 * o.G / acc : 0.0;
    }
}

__global__ void __launch_bounds__(256) k_osb_dilation(const StepArgsF64 a, OsbArgs o)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const double2* __restrict__ rin = reinterpret_cast<const double2*>(a.rec[step & 1]);
    const int64_t W = 32LL * a.Q;
    const int64_t nslices = (a.n + 31) >> 5;
    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int64_t i = (g << 5) + lane;
        const int Wg = a.sw[g];
        double acc = 0.0;
        for (int q = 0; q * 32 < Wg; ++q) {
            uint32_t* bw = a.bits + (g * a.Q + q) * 32 + lane;
            const uint32_t word = *bw;
            uint32_t nword = word;
            const int mend = min(32, Wg - q * 32);
            for (int b = 0; b < mend; ++b) {
                if (!((word >> b) & 1u)) continue;
                const int64_t slot = (g * W + q * 32 + b) * 32 + lane;
                const int64_t j = a.nbr[slot];
                const OsbBond bd = osb_bond(rin, i, j);
                const double L = o.len[slot];
                const double e = bd.r - L;
                const double s = e * a.ilen[slot];
                bool brk = !a.frozen && s >= bond_sc(a, i, j);
                if (brk && a.has_nofail)
                    brk = ((a.bct[a.bcc[i]].mask | a.bct[a.bcc[j]].mask) & 8u) == 0u;
                if (brk) {
                    nword &= ~(1u << b);
                    continue;
                }
                acc += L * e * o.vol[j];
            }
            if (nword != word) *bw = nword;
        }
        const double m = o.mvol[i];
        const double th = m > 0.0 ? 3.0 * acc / m : 0.0;
        o.theta[i] = th;
        o.alpha[i] = m > 0.0 ? 3.0 * o.K * th / m - o.beta[i] * th / 3.0 : 0.0;
    }
}

__global__ void __launch_bounds__(256) k_osb_force(const StepArgsF64 a, OsbArgs o)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const int cur = (int)(step & 1);
    const double2* __restrict__ rin = reinterpret_cast<const double2*>(a.rec[cur]);
    double2* __restrict__ rout = reinterpret_cast<double2*>(const_cast<double*>(a.rec[cur ^ 1]));
    const int64_t W = 32LL * a.Q;
    const int64_t nslices = (a.n + 31) >> 5;
    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int64_t i = (g << 5) + lane;
        const int Wg = a.sw[g];
        const double ai = o.alpha[i], bi = o.beta[i];
        double fx = 0.0, fy = 0.0, fz = 0.0, ws = 0.0;
        for (int q = 0; q * 32 < Wg; ++q) {
            const uint32_t word = a.bits[(g * a.Q + q) * 32 + lane];
            const int mend = min(32, Wg - q * 32);
            for (int b = 0; b < mend; ++b) {
                if (!((word >> b) & 1u)) continue;
                const int64_t slot = (g * W + q * 32 + b) * 32 + lane;
                const int64_t j = a.nbr[slot];
                const OsbBond bd = osb_bond(rin, i, j);
                const double L = o.len[slot];
                const double e = bd.r - L;
                // t_ij + t_ji
                const double t = (ai + o.alpha[j]) * L + (bi + o.beta[j]) * e;
                const double f = t * o.vol[j] * bd.ir;
                fx += f * bd.y0;
                fy += f * bd.y1;
                fz += f * bd.y2;
                ws += __ldg(reinterpret_cast<const double*>(rin) + 8 * j + 3);
            }
        }
        if (i >= a.n) continue;
        // damped Euler-Cromer update, boundary conditions and damage (as the
        // bond-based FP64 step)
        const double2 x01 = rin[4 * i], x23 = rin[4 * i + 1], u01 = rin[4 * i + 2],
                      u23 = rin[4 * i + 3];
        const uint32_t cls = a.bcc[i];
        uint32_t mask = 0u;
        double gdisp[3] = {0.0, 0.0, 0.0};
        double F[3] = {fx, fy, fz};
        if (cls != 0u) {
            const BcClass& bc = a.bct[cls];
            mask = bc.mask;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                gdisp[c] = bc.disp[c];
                F[c] += a.load * bc.force[c];
            }
        }
        const double s_now = bc_scale(a.disp_rate, a.ramp_steps, step);
        const double s_next = bc_scale(a.disp_rate, a.ramp_steps, step + 1);
        const double uo[3] = {u01.x, u01.y, u23.x};
        // velocity-Verlet: a^n is formed afresh at the step the state was set
        const bool first = a.vv && step == a.step_ctr[1];
        double un[3];
        bool finite = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // stored velocity: v^n (Euler-Cromer) or the half-step velocity
            // (velocity-Verlet), as in the bond-based FP64 step
            const double vi = a.v[3 * i + c];
            double vn, vfull;
            if (a.vv) {
                const double acc = (F[c] - a.eta * vi) / a.rho;
                vfull = first ? vi : vi + 0.5 * a.dt * acc;
                vn = vfull + 0.5 * a.dt * acc;
            } else {
                vn = vi + a.dt * (F[c] - a.eta * vi) / a.rho;
                vfull = vn;
            }
            double u = uo[c] + a.dt * vn;
            if (mask & (1u << c)) {
                u = gdisp[c] * s_next;
                vn = gdisp[c] * (s_next - s_now) / a.dt;
                vfull = vi;
            }
            finite = finite && isfinite(u);
            un[c] = u;
            if (a.peek)
                a.vout[3 * i + c] = vfull;
            else
                a.v[3 * i + c] = vn;
        }
        if (a.peek) continue;  // the read-only force pass of velocity-Verlet
        rout[4 * i] = x01;
        rout[4 * i + 1] = x23;
        rout[4 * i + 2] = make_double2(un[0], un[1]);
        rout[4 * i + 3] = make_double2(un[2], 0.0);
        const double wi = a.wsum_inv[i];
        a.damage[i] = wi > 0.0 ? fmax(0.0, 1.0 - ws * wi) : 0.0;
        if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
    }
}

__global__ void k_osb_len(const double* __restrict__ x64, const int32_t* __restrict__ nbr,
                          const int32_t* __restrict__ sw, int64_t n, int Q, double* __restrict__ len)
{
    const int64_t W = 32LL * Q;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < (((n + 31) >> 5) << 5);
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = p >> 5;
        const int lane = (int)(p & 31);
        for (int m = 0; m < sw[g]; ++m) {
            const int64_t slot = (g * W + m) * 32 + lane;
            const int64_t j = nbr[slot];
            double v = 0.0;
            if (j != p) {
                const double e0 = x64[3 * j] - x64[3 * p], e1 = x64[3 * j + 1] - x64[3 * p + 1],
                             e2 = x64[3 * j + 2] - x64[3 * p + 2];
                v = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
            }
            len[slot] = v;
        }
    }
}

int grid_nodes(int64_t n)
{
    int64_t g = ((((n + 31) >> 5) << 5) + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 65535 * 8 ? 65535 * 8 : g));
}

}  // namespace

cudaError_t launch_osb_setup(const StepArgsF64& a, const OsbArgs& o, const double* x64,
                             cudaStream_t s)
{
    k_osb_len<<<grid_nodes(a.n), 256, 0, s>>>(x64, a.nbr, a.sw, a.n, a.Q, o.len);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_osb_weighted_volume<<<grid_nodes(a.n), 256, 0, s>>>(a, o);
    return cudaGetLastError();
}

cudaError_t launch_osb_step(const StepArgsF64& a, const OsbArgs& o, int grid, int block,
                            cudaStream_t s)
{
    k_osb_dilation<<<grid, block, 0, s>>>(a, o);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_osb_force<<<grid, block, 0, s>>>(a, o);
    return cudaGetLastError();
}

}  // namespace pd
