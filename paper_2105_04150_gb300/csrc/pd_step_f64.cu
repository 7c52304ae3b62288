// Fused FP64 peridynamic step kernel for sm_103a (the parity path).
//
// Same decomposition as the FP32-bulk kernel (lane per node over the sliced
// family layout, double-buffered displacement, bond flags as the lane's own
// bit words, integration and damage in the same pass), but every quantity is
// FP64 and the stretch is that of Eq. 4, s = (|xi + eta| - |xi|) / |xi|, so
// break decisions are FP64 decisions.  GB300's FP64 rate is a small fraction
// of its FP32 rate and this kernel is bound by it, so the per-bond square roots
// and divisions are avoided: 1/|xi| is a per-slot array computed once (8 bytes
// per bond: memory is not the limit here), and 1/|y| comes from a Newton-
// refined reciprocal square root; then |y| = |y|^2 / |y|, s = |y| / |xi| - 1
// (one rounding, an absolute error of a few 1e-16) and the force scale is
// c V s / |y| with multiplications only.
// Node record: 8 doubles {x, y, z, w, ux, uy, uz, 0}, w = c V (or V with
// per-bond stiffness).
#include <cuda_runtime.h>

#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kUnroll = 2;

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

template <int SCM>
__global__ void __launch_bounds__(256) k_step_f64(const StepArgsF64 a)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const bool first = a.vv && step == a.step_ctr[1];  // velocity-Verlet: a^n formed afresh
    const int cur = (int)(step & 1);
    const int Q = a.Q;
    const int64_t W = 32LL * Q;
    const int64_t nslices = (a.n + 31) >> 5;
    const double2* __restrict__ rin = reinterpret_cast<const double2*>(a.rec[cur]);
    double2* __restrict__ rout = reinterpret_cast<double2*>(const_cast<double*>(a.rec[cur ^ 1]));
    const double* __restrict__ cb = a.cbond;

    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int64_t i = (g << 5) + lane;
        const int Wg = a.sw[g];
        const double2 x01 = __ldg(rin + 4 * i), x23 = __ldg(rin + 4 * i + 1);
        const double2 u01 = __ldg(rin + 4 * i + 2), u23 = __ldg(rin + 4 * i + 3);
        const int32_t* __restrict__ col = a.nbr + g * W * 32 + lane;
        uint32_t* bw = a.bits + g * Q * 32 + lane;
        double fx = 0.0, fy = 0.0, fz = 0.0, ws = 0.0;

        for (int q = 0; q * 32 < Wg; ++q) {
            const uint32_t word = bw[q * 32];
            uint32_t nword = word;
            const int mend = min(32, Wg - q * 32);
            for (int b0 = 0; b0 < mend; b0 += kUnroll) {
                int32_t jj[kUnroll];
                bool al[kUnroll];
                double2 ra[kUnroll][4];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const int b = b0 + u;
                    al[u] = (b < mend) && ((word >> b) & 1u);
                    jj[u] = al[u] ? __ldg(col + (int64_t)(q * 32 + b) * 32) : 0;
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u)
                    if (al[u])
#pragma unroll
                        for (int e = 0; e < 4; ++e) ra[u][e] = __ldg(rin + 4 * (int64_t)jj[u] + e);
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    if (!al[u]) continue;
                    const double ex = ra[u][0].x - x01.x, ey = ra[u][0].y - x01.y;
                    const double ez = ra[u][1].x - x23.x;
                    const double yx = ex + (ra[u][2].x - u01.x);
                    const double yy = ey + (ra[u][2].y - u01.y);
                    const double yz = ez + (ra[u][3].x - u23.x);
                    const int64_t slot = (g * W + q * 32 + b0 + u) * 32 + lane;
                    const double y2 = yx * yx + yy * yy + yz * yz;
                    const double ir = rsqrt_nr(y2);
                    const double r = y2 * ir;
                    const double s = fma(r, __ldg(a.ilen + slot), -1.0);
                    double sc;
                    if (a.inst != nullptr) {  // batch: instance parameters, local ids as keys
                        const InstParams& ip = a.itab[a.inst[i]];
                        sc = ip.sc_mode == 1 ? sc_draw(ip.sc_seed, ip.sc_lo, ip.sc_hi, a.hid[i],
                                                       a.hid[jj[u]])
                                             : ip.sc;
                    } else {
                        sc = (SCM == 0) ? a.sc
                                        : sc_draw(a.sc_seed, a.sc_lo, a.sc_hi, a.gid[i],
                                                  a.gid[jj[u]]);
                    }
                    bool brk = !a.frozen && s >= sc;
                    if (brk && a.has_nofail) brk = !pair_no_fail(a.bcc, a.bct, i, jj[u]);
                    if (brk) {
                        nword &= ~(1u << (b0 + u));
                        if (a.integ != nullptr) a.integ[slot] = 0.0;
                    } else {
                        // bilinear softening: the integrity only decreases, as the
                        // stretch passes s_0 = s_c / kr (a no-fail bond past s_c keeps 0)
                        double mu = 1.0;
                        if (a.integ != nullptr) {
                            mu = a.integ[slot];
                            const double s0 = sc / a.kr;
                            if (s > s0) {
                                const double ms =
                                    s >= sc ? 0.0 : soft_mu_of(s, s0, sc, a.k1, a.beta);
                                if (ms < mu) {
                                    mu = ms;
                                    a.integ[slot] = ms;
                                }
                            }
                        }
                        double wj = ra[u][1].y * mu;
                        if (cb != nullptr) wj *= __ldg(cb + slot);
                        const double f = wj * s * ir;
                        fx += f * yx;
                        fy += f * yy;
                        fz += f * yz;
                        ws += ra[u][1].y * mu;
                    }
                }
            }
            if (nword != word) bw[q * 32] = nword;
        }

        if (i < a.n) {
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
            double un[3];
            bool finite = true;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // stored velocity: v^n (Euler-Cromer) or, for velocity-Verlet, the
                // half-step velocity v^{n-1} + dt/2 a^{n-1} (v^n right after a set state)
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
            if (a.peek) continue;
            rout[4 * i] = x01;
            rout[4 * i + 1] = x23;
            rout[4 * i + 2] = make_double2(un[0], un[1]);
            rout[4 * i + 3] = make_double2(un[2], 0.0);
            const double wi = a.wsum_inv[i];
            // clamp: ws * (1 / sum w) can round to 1 + 1 ulp for an intact family
            a.damage[i] = wi > 0.0 ? fmax(0.0, 1.0 - ws * wi) : 0.0;
            if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
        }
    }
}

}  // namespace

cudaError_t launch_step_f64(const StepArgsF64& a, int sc_mode, int grid, int block, cudaStream_t s)
{
    if (sc_mode == 0)
        k_step_f64<0><<<grid, block, 0, s>>>(a);
    else
        k_step_f64<1><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

const void* step_f64_kernel(int sc_mode)
{
    return sc_mode == 0 ? (const void*)k_step_f64<0> : (const void*)k_step_f64<1>;
}

}  // namespace pd
