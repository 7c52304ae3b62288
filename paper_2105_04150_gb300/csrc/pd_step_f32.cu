// Fused FP32-bulk peridynamic step kernel for sm_103a.
//
// One launch = one explicit time step: bond kinematics (Eq. 4), irreversible
// breaking (Eq. 6), pairwise PMB force (Eq. 5) reduced onto the node
// (Eq. 10), body force, damped Euler-Cromer update (Eq. 11), displacement
// BCs and damage (Eq. 8).  The paper splits this into a bond kernel and an
// integrator kernel because an in-place update would race with neighbours
// still reading u^n (Section 3.3); here the displacement that neighbours read
// is double-buffered (step k reads buffer k&1, writes (k+1)&1), so the whole
// step is one kernel and every node's data crosses HBM once per step.
//
// Work decomposition ("lane per node" over a sliced ELL): a warp owns a slice
// of 32 consecutive nodes and walks their families in lockstep, slot m of all
// 32 nodes per iteration - one coalesced 128-byte load of neighbour ids - so
// each lane accumulates its own node's force in registers: no shared-memory
// reduction, no shuffles, no barriers.  Bond flags are the lane's own 32-bit
// words.  The slot loop is branch-free: slots beyond a lane's family or of
// broken bonds are evaluated and masked (the paper's thread-divergence
// trade-off, Section 3.5, resolved in favour of no divergence at all, with the
// padding bounded per slice instead of per power of two).  The slice's
// neighbour-id block is requested from HBM with one bulk L2 prefetch when the
// warp starts it, so the stream does not wait for the warp's own loads.
// Each node's gather data is one 48-byte record {x~, w | h | l}.
//
// Precision: bond arithmetic is FP32 in units of the horizon with the
// cancellation-free stretch s = eta.(2 xi + eta) / (|xi| (|xi| + |xi+eta|)).
// The displacement is an unevaluated float-float sum h + l (48-bit
// significand): it is accumulated exactly enough by two-sum updates and gives
// eta = (h_j - h_i) + (l_j - l_i) to FP32 relative accuracy even when |u| is
// far larger than |eta|.  The arithmetic is exactly antisymmetric (bond j->i
// sees -xi, -eta and produces the same bits), so both directions of a bond
// break together.  A bond whose FP32 stretch lies within a relative band of
// s_c is re-tested with the literal FP64 stretch of Eq. 4.
#include <cuda_runtime.h>

#include "pd_internal.h"

namespace pd {
namespace {

#ifndef PD_F32_UNROLL
#define PD_F32_UNROLL 4
#endif
#ifndef PD_F32_MIN_BLOCKS
#define PD_F32_MIN_BLOCKS 3
#endif
constexpr int kUnroll = PD_F32_UNROLL;  // family slots in flight per lane

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

__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// (s, e) = exact sum of a and b (Knuth's two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// h + l += d, keeping |l| <= ulp(h)/2.
__device__ __forceinline__ void ff_add(float& h, float& l, float d)
{
    float s, e;
    two_sum(h, d, s, e);
    e += l;
    h = s + e;
    l = e - (h - s);
}

__device__ __forceinline__ void ff_set(double x, float& h, float& l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

// FP32 bond kinematics in horizon units: y = xi + eta, num = eta.(2 xi + eta)
// = |y|^2 - |xi|^2 (no cancellation), den = |xi| (|xi| + |y|), so s = num / den.
struct BondF32 {
    float yx, yy, yz, num, den, y2;
};

__device__ __forceinline__ BondF32 bond_f32(const float4 xi, const float4 hi, const float2 li,
                                            const float4 xj, const float4 hj, const float2 lj)
{
    BondF32 r;
    const float ex = xj.x - xi.x, ey = xj.y - xi.y, ez = xj.z - xi.z;
    const float hx = (hj.x - hi.x) + (hj.w - hi.w);
    const float hy = (hj.y - hi.y) + (lj.x - li.x);
    const float hz = (hj.z - hi.z) + (lj.y - li.y);
    r.yx = ex + hx;
    r.yy = ey + hy;
    r.yz = ez + hz;
    const float xx = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
    r.num = fmaf(hx, ex + r.yx, fmaf(hy, ey + r.yy, hz * (ez + r.yz)));
    r.y2 = xx + r.num;
    const float p = xx * r.y2;
    r.den = xx + p * rsqrtf(p);
    return r;
}

// c V_j s / |y| = w num / (den |y|)
__device__ __forceinline__ float bond_coef(const BondF32& b, float w)
{
    return w * b.num * rsqrtf(b.den * b.den * b.y2);
}

// A bond whose FP32 stretch reached the band just below the smallest s_c: the
// break test is decided in FP32 when s is clearly away from the bond's s_c and
// otherwise with the literal FP64 stretch of Eq. 4 (FP64 positions, float-float
// displacement); the no-fail rule applies last.  Returns the bond's force
// contribution {fx, fy, fz, w}, all zero when it breaks (*broken = true).
template <int SCM>
__device__ __noinline__ float4 resolve_bond(const StepArgsF32& a, int cur, int64_t i, int64_t j,
                                            int64_t slot, bool* broken)
{
    const float4* __restrict__ R = a.rec[cur];
    const float4 xi = R[3 * i], hi = R[3 * i + 1], xj = R[3 * j], hj = R[3 * j + 1];
    const float2 li = *reinterpret_cast<const float2*>(R + 3 * i + 2);
    const float2 lj = *reinterpret_cast<const float2*>(R + 3 * j + 2);
    const BondF32 b = bond_f32(xi, hi, li, xj, hj, lj);
    double sc = a.sc;
    float scf = a.sc_f;
    if (SCM == 1) {
        sc = sc_draw(a.sc_seed, a.sc_lo, a.sc_hi, a.gid[i], a.gid[j]);
        scf = (float)sc;
    }
    const float r = fmaf(-scf, b.den, b.num);  // den * (s - s_c)
    bool brk;
    if (fabsf(r) > a.guard * scf * b.den) {
        brk = r >= 0.0f;
    } else {
        const double ui[3] = {(double)hi.x + (double)hi.w, (double)hi.y + (double)li.x,
                              (double)hi.z + (double)li.y};
        const double uj[3] = {(double)hj.x + (double)hj.w, (double)hj.y + (double)lj.x,
                              (double)hj.z + (double)lj.y};
        double xv[3], y[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xv[c] = a.x64[3 * j + c] - a.x64[3 * i + c];
            y[c] = xv[c] + (uj[c] - ui[c]) * a.delta;
        }
        const double L = sqrt(xv[0] * xv[0] + xv[1] * xv[1] + xv[2] * xv[2]);
        const double Rr = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
        brk = (Rr - L) / L >= sc;
    }
    if (brk && a.has_nofail) brk = ((a.bct[a.bcc[i]].mask | a.bct[a.bcc[j]].mask) & 8u) == 0u;
    *broken = brk;
    if (brk) return make_float4(0.f, 0.f, 0.f, 0.f);
    float w = xj.w;
    if (a.cbond != nullptr) w *= a.cbond[slot];
    const float coef = bond_coef(b, w);
    return make_float4(coef * b.yx, coef * b.yy, coef * b.yz, xj.w);
}

template <int SCM>
__global__ void __launch_bounds__(256, PD_F32_MIN_BLOCKS) k_step_f32(const __grid_constant__ StepArgsF32 a)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = *a.step_ctr + a.k;
    const int cur = (int)(step & 1);
    const int Q = a.Q;
    const int64_t W = 32LL * Q;
    const int64_t nslices = (a.n + 31) >> 5;
    const float4* __restrict__ R = a.rec[cur];
    float4* __restrict__ Rout = const_cast<float4*>(a.rec[cur ^ 1]);
    const float* __restrict__ cb = a.cbond;
    const float fast_lo = a.fast_lo;

    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int Wg = a.sw[g];
        const int32_t* __restrict__ col = a.nbr + g * W * 32 + lane;
        if (lane == 0) prefetch_l2(col, (uint32_t)(((Wg + 3) & ~3) * 128));
        const int64_t i = (g << 5) + lane;
        const float4 xi = __ldg(R + 3 * i);
        const float4 hi = __ldg(R + 3 * i + 1);
        const float2 li = __ldg(reinterpret_cast<const float2*>(R + 3 * i + 2));
        uint32_t* bw = a.bits + g * Q * 32 + lane;
        float fx = 0.f, fy = 0.f, fz = 0.f, ws = 0.f;

        for (int q = 0; q * 32 < Wg; ++q) {
            const uint32_t word = bw[q * 32];
            uint32_t nword = word;
            uint32_t pend = 0u;  // members in the near-s_c band, resolved below
            const int mend = min(32, Wg - q * 32);
            const int32_t* __restrict__ cq = col + (int64_t)q * 32 * 32;
            for (int b0 = 0; b0 < mend; b0 += kUnroll) {
                // every slot is evaluated; slots that are broken or unused (their
                // id is the node itself) are masked out with selects, so the warp
                // never diverges in this loop
                int32_t jj[kUnroll];
                float4 xa[kUnroll], ha[kUnroll];
                float2 la[kUnroll];
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) jj[u] = __ldg(cq + (b0 + u) * 32);
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const float4* rj = R + 3 * (int64_t)jj[u];
                    xa[u] = __ldg(rj);
                    ha[u] = __ldg(rj + 1);
                    la[u] = __ldg(reinterpret_cast<const float2*>(rj + 2));
                }
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const bool alive = (word >> (b0 + u)) & 1u;
                    const BondF32 bd = bond_f32(xi, hi, li, xa[u], ha[u], la[u]);
                    const bool cand = alive && (bd.num >= fast_lo * bd.den);
                    const bool take = alive && !cand;
                    pend |= cand ? (1u << (b0 + u)) : 0u;
                    float wj = xa[u].w;
                    if (cb != nullptr) wj *= __ldg(cb + (g * W + q * 32 + b0 + u) * 32 + lane);
                    float coef = bond_coef(bd, wj);
                    coef = take ? coef : 0.0f;
                    fx = fmaf(coef, bd.yx, fx);
                    fy = fmaf(coef, bd.yy, fy);
                    fz = fmaf(coef, bd.yz, fz);
                    ws += take ? xa[u].w : 0.0f;
                }
            }
            while (pend) {
                const int b = __ffs(pend) - 1;
                pend &= pend - 1u;
                const int64_t slot = (g * W + q * 32 + b) * 32 + lane;
                bool broken;
                const float4 f = resolve_bond<SCM>(a, cur, i, cq[b * 32], slot, &broken);
                if (broken) {
                    nword &= ~(1u << b);
                } else {
                    fx += f.x;
                    fy += f.y;
                    fz += f.z;
                    ws += f.w;
                }
            }
            if (nword != word) bw[q * 32] = nword;
        }

        // ---- integration of the lane's node (Eq. 11, damped Euler-Cromer)
        if (i < a.n) {
            const uint32_t cls = a.bcc[i];
            uint32_t mask = 0u;
            const BcClass* bc = nullptr;
            float F[3] = {fx, fy, fz};
            if (cls != 0u) {
                bc = a.bct + cls;
                mask = bc->mask;
#pragma unroll
                for (int c = 0; c < 3; ++c) F[c] += (float)(a.load * bc->force[c]);
            }
            const float dtf = (float)a.dt, etaf = (float)a.eta, rhof = (float)a.rho;
            const float dtd = (float)(a.dt * a.inv_delta);
            float H[3] = {hi.x, hi.y, hi.z};
            float L[3] = {hi.w, li.x, li.y};
            bool finite = true;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float vi = a.v[3 * i + c];
                float vn = vi + dtf * (F[c] - etaf * vi) / rhof;
                ff_add(H[c], L[c], vn * dtd);
                if (mask & (1u << c)) {
                    const double s_now = a.disp_rate * (double)step;
                    const double s_next = a.disp_rate * (double)(step + 1);
                    ff_set(bc->disp[c] * s_next * a.inv_delta, H[c], L[c]);
                    vn = (float)(bc->disp[c] * (s_next - s_now) / a.dt);
                }
                finite = finite && isfinite(H[c]);
                a.v[3 * i + c] = vn;
            }
            Rout[3 * i] = xi;
            Rout[3 * i + 1] = make_float4(H[0], H[1], H[2], L[0]);
            Rout[3 * i + 2] = make_float4(L[1], L[2], 0.0f, 0.0f);
            const float wi = a.wsum_inv[i];
            a.damage[i] = wi > 0.0f ? 1.0f - ws * wi : 0.0f;
            if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
        }
    }
}

}  // namespace

cudaError_t launch_step_f32(const StepArgsF32& a, int sc_mode, int grid, int block, cudaStream_t s)
{
    if (sc_mode == 0)
        k_step_f32<0><<<grid, block, 0, s>>>(a);
    else
        k_step_f32<1><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

const void* step_f32_kernel(int sc_mode)
{
    return sc_mode == 0 ? (const void*)k_step_f32<0> : (const void*)k_step_f32<1>;
}

}  // namespace pd
