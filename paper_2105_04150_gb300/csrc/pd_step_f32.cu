// Fused FP32-bulk peridynamic step kernel for sm_103a.
//
// One launch = one explicit time step (bond kinematics, irreversible breaking,
// force reduction, body force, damped Euler-Cromer update, displacement BCs,
// damage), i.e. the bond-force + reduction kernel and the integrator kernel of
// the paper (Algorithm bond_index, Algorithm reduction, Section 3.3) fused
// into one pass.  The paper keeps integration in a second kernel because an
// in-place update would race with neighbours still reading u^n (Section 3.3);
// here every array that neighbours read (node records, FP64 displacement) is
// double-buffered, so step k reads buffer k&1 and writes buffer (k+1)&1.
//
// Work decomposition: a warp owns a group of 32 consecutive nodes (spatial
// order).  For each node of the group, lane l evaluates the family members
// q*32+l (q < Q) - one coalesced 128-byte load of neighbour ids per q - and the
// four partial sums (force x/y/z and intact-bond weight) are reduced with a
// shuffle butterfly; lane t keeps node t's totals.  The group's integration
// then runs lane-parallel (lane t integrates node t) with coalesced node loads
// and stores.  Bond flags are bits: word q of a node is exactly the ballot of
// its lanes' "still intact" predicates for round q.
//
// Precision: bond arithmetic is FP32 in units of the horizon, using the
// cancellation-free stretch s = eta.(2 xi + eta) / (|xi| (|xi| + |xi+eta|)).
// It is exactly antisymmetric: bond j->i sees -xi, -eta and computes the same
// bits as i->j, so both directions break together.  A bond whose FP32 stretch
// lies within a relative band `guard` of s_c is re-tested with the literal
// FP64 stretch of Eq. 4 from FP64 positions and displacements, so the break
// decision is the FP64 one.  Displacements accumulate in FP64.
#include <cuda_runtime.h>

#include "pd_internal.h"

namespace pd {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output m of the stream seeded
// with `seed`.  Used as a counter-based draw of the per-bond critical stretch.
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

// Literal FP64 stretch of Eq. 4 for the bond i->j and the break test of Eq. 6.
__device__ __noinline__ bool retest_f64(const double* __restrict__ x64,
                                        const double* __restrict__ u, int64_t i, int64_t j,
                                        double sc)
{
    double xi[3], y[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xi[c] = x64[3 * j + c] - x64[3 * i + c];
        y[c] = xi[c] + (u[3 * j + c] - u[3 * i + c]);
    }
    const double L = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    const double r = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
    return (r - L) / L >= sc;
}

__device__ __noinline__ bool pair_no_fail(const uint8_t* __restrict__ bcc,
                                          const BcClass* __restrict__ bct, int64_t i, int64_t j)
{
    return ((bct[bcc[i]].mask | bct[bcc[j]].mask) & 8u) != 0u;
}

// Break decision for an intact bond with FP32 stretch num/den (den > 0).
template <int SCM>
__device__ __forceinline__ bool decide_break(const StepArgsF32& a, const double* __restrict__ uin,
                                             int64_t i, int64_t j, float num, float den)
{
    if (SCM == 0) {
        const float r = fmaf(-a.sc_f, den, num);  // sign of s - s_c
        if (fabsf(r) > a.guard * a.sc_f * den) return r >= 0.0f;
        return retest_f64(a.x64, uin, i, j, a.sc);
    } else {
        // s_c in [sc_lo, sc_hi): most bonds are clearly below sc_lo.
        const float rlo = fmaf(-a.sc_lo_f, den, num);
        if (rlo < -a.guard * a.sc_lo_f * den) return false;
        const double sc = sc_draw(a.sc_seed, a.sc_lo, a.sc_hi, a.gid[i], a.gid[j]);
        const float scf = (float)sc;
        const float r = fmaf(-scf, den, num);
        if (fabsf(r) > a.guard * scf * den) return r >= 0.0f;
        return retest_f64(a.x64, uin, i, j, sc);
    }
}

template <int QT, int SCM>
__global__ void __launch_bounds__(256) k_step_f32(const StepArgsF32 a)
{
    const int Q = (QT > 0) ? QT : a.q_rt;
    const int W = 32 * Q;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = *a.step_ctr + a.k;
    const int cur = (int)(step & 1);
    const float4* __restrict__ rin = a.rec[cur];
    float4* __restrict__ rout = const_cast<float4*>(a.rec[cur ^ 1]);
    const double* __restrict__ uin = a.u64[cur];
    double* __restrict__ uout = a.u64[cur ^ 1];
    const float* __restrict__ cb = a.cbond;
    const int64_t ngroups = (a.n + 31) >> 5;

    for (int64_t g = wid; g < ngroups; g += nwarps) {
        const int64_t base = g << 5;
        const int cnt = (int)min((int64_t)32, a.n - base);
        float kx = 0.f, ky = 0.f, kz = 0.f, kw = 0.f;

        for (int t = 0; t < cnt; ++t) {
            const int64_t i = base + t;
            const float4 xi = __ldg(rin + 2 * i);
            const float4 ui = __ldg(rin + 2 * i + 1);
            const int32_t* __restrict__ row = a.nbr + i * W;
            uint32_t* brow = a.bits + i * Q;
            float fx = 0.f, fy = 0.f, fz = 0.f, ws = 0.f;

            for (int q0 = 0; q0 < Q; q0 += 4) {
                uint32_t w[4];
                int32_t jj[4];
                bool al[4];
                float4 xa[4], ua[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
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
                for (int c = 0; c < 4; ++c) {
                    if (al[c]) {
                        xa[c] = __ldg(rin + 2 * (int64_t)jj[c]);
                        ua[c] = __ldg(rin + 2 * (int64_t)jj[c] + 1);
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (al[c]) {
                        const float ex = xa[c].x - xi.x, ey = xa[c].y - xi.y, ez = xa[c].z - xi.z;
                        const float hx = ua[c].x - ui.x, hy = ua[c].y - ui.y, hz = ua[c].z - ui.z;
                        const float yx = ex + hx, yy = ey + hy, yz = ez + hz;
                        const float xx = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                        // eta . (2 xi + eta) = |y|^2 - |xi|^2 without cancellation
                        const float num = fmaf(hx, ex + yx, fmaf(hy, ey + yy, hz * (ez + yz)));
                        const float y2 = xx + num;
                        const float p = xx * y2;
                        const float lxly = p * rsqrtf(p);           // |xi| |y|
                        const float den = xx + lxly;                 // |xi| (|xi| + |y|)
                        bool brk = decide_break<SCM>(a, uin, i, jj[c], num, den);
                        if (brk && a.has_nofail) brk = !pair_no_fail(a.bcc, a.bct, i, jj[c]);
                        if (brk) {
                            al[c] = false;
                        } else {
                            // c V_j s / |y| = w_j num / (den |y|)
                            float wj = xa[c].w;
                            if (cb != nullptr) wj *= __ldg(cb + i * W + (q0 + c) * 32 + lane);
                            const float coef = wj * num * rsqrtf(den * den * y2);
                            fx = fmaf(coef, yx, fx);
                            fy = fmaf(coef, yy, fy);
                            fz = fmaf(coef, yz, fz);
                            ws += xa[c].w;
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
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

        // ---- lane-parallel integration of the group (Eq. 11, damped Euler-Cromer)
        if (lane < cnt) {
            const int64_t i = base + lane;
            const uint32_t cls = a.bcc[i];
            uint32_t mask = 0u;
            double gdisp[3] = {0.0, 0.0, 0.0};
            float F[3] = {kx, ky, kz};
            if (cls != 0u) {
                const BcClass& bc = a.bct[cls];
                mask = bc.mask;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    gdisp[c] = bc.disp[c];
                    F[c] += (float)(a.load * bc.force[c]);
                }
            }
            const double s_now = a.disp_rate * (double)step;
            const double s_next = a.disp_rate * (double)(step + 1);
            const float dtf = (float)a.dt, etaf = (float)a.eta, rhof = (float)a.rho;
            double un[3];
            bool finite = true;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float vi = a.v[3 * i + c];
                float vn = vi + dtf * (F[c] - etaf * vi) / rhof;
                double u = uin[3 * i + c] + a.dt * (double)vn;
                if (mask & (1u << c)) {
                    u = gdisp[c] * s_next;
                    vn = (float)(gdisp[c] * (s_next - s_now) / a.dt);
                }
                finite = finite && isfinite(u);
                un[c] = u;
                a.v[3 * i + c] = vn;
                uout[3 * i + c] = u;
            }
            rout[2 * i] = __ldg(rin + 2 * i);
            rout[2 * i + 1] = make_float4((float)(un[0] * a.inv_delta), (float)(un[1] * a.inv_delta),
                                          (float)(un[2] * a.inv_delta), 0.0f);
            a.damage[i] = 1.0f - kw * a.wsum_inv[i];
            if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
        }
    }
}

template <int QT>
cudaError_t launch_q(const StepArgsF32& a, int sc_mode, int grid, int block, cudaStream_t s)
{
    if (sc_mode == 0)
        k_step_f32<QT, 0><<<grid, block, 0, s>>>(a);
    else
        k_step_f32<QT, 1><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int QT>
const void* kernel_ptr(int sc_mode)
{
    return sc_mode == 0 ? (const void*)k_step_f32<QT, 0> : (const void*)k_step_f32<QT, 1>;
}

}  // namespace

cudaError_t launch_step_f32(const StepArgsF32& a, int Q, int sc_mode, int grid, int block,
                            cudaStream_t s)
{
    switch (Q) {
        case 4: return launch_q<4>(a, sc_mode, grid, block, s);
        case 5: return launch_q<5>(a, sc_mode, grid, block, s);
        default: return launch_q<0>(a, sc_mode, grid, block, s);
    }
}

const void* step_f32_kernel(int Q, int sc_mode)
{
    switch (Q) {
        case 4: return kernel_ptr<4>(sc_mode);
        case 5: return kernel_ptr<5>(sc_mode);
        default: return kernel_ptr<0>(sc_mode);
    }
}

}  // namespace pd
