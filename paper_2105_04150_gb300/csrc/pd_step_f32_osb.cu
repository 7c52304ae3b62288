// State-based build of the FP32 kernels: the ordinary state-based model's
// dilation and force kernels over the bond-based step's records and helpers,
// which this translation unit takes from pd_step_f32.cu (see PD_F32_OSB there).
#define PD_F32_OSB 1
#include "pd_step_f32.cu"

namespace pd {
namespace {
// ---------------------------------------------------------------------------
// Ordinary state-based model in FP32 (the FP64 form and the formulas are in
// pd_step_osb.cu).  Lengths in horizon units: e = |y| - |xi| comes out of the
// cancellation-free bond terms as num |xi| / den (den = |xi| (|xi| + |y|)), so
// the dilation's |xi| e = num |xi|^2 / den needs no length at all and the force
// forms |xi| from |xi|^2 with one reciprocal square root: no per-slot length
// is stored or read.  theta is unit free; the per-node coefficients are stored
// multiplied by delta (alpha' = delta alpha, beta' = delta beta with m in
// horizon units) as one (alpha', beta') pair per node, so that
// t'_ij + t'_ji = (alpha'_i + alpha'_j) |xi| + (beta'_i + beta'_j) e is a force
// density per unit volume.  Bonds break in the dilation kernel, with the
// near-s_c decision of the bond-based kernel; node weights are the volumes.

__device__ __forceinline__ void integrate_osb_f32(const StepArgsF32& a, int64_t i, int64_t step,
                                                  float fx, float fy, float fz, float ws,
                                                  const NodeF32& ni, float4* Rout)
{
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
    const float4 lo = a.lo32[i];
    float H[3] = {ni.hx, ni.hy, ni.hz};
    float L[3] = {lo.x, lo.y, lo.z};
    // velocity-Verlet: a^n is formed afresh at the step the state was set
    const bool first = a.vv && step == a.step_ctr[1];
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        // stored velocity: v^n (Euler-Cromer) or the half-step velocity
        // (velocity-Verlet), as in the bond-based FP32 step
        const float vi = a.v[3 * i + c];
        float vn, vfull;
        if (a.vv) {
            const float acc = (F[c] - etaf * vi) / rhof;
            vfull = first ? vi : vi + 0.5f * dtf * acc;
            vn = vfull + 0.5f * dtf * acc;
        } else {
            vn = vi + dtf * (F[c] - etaf * vi) / rhof;
            vfull = vn;
        }
        ff_add(H[c], L[c], vn * dtd);
        if (mask & (1u << c)) {
            const double s_now = bc_scale(a.disp_rate, a.ramp_steps, step);
            const double s_next = bc_scale(a.disp_rate, a.ramp_steps, step + 1);
            ff_set(bc->disp[c] * s_next * a.inv_delta, H[c], L[c]);
            vn = (float)(bc->disp[c] * (s_next - s_now) / a.dt);
            vfull = vi;
        }
        finite = finite && isfinite(H[c]);
        if (a.peek)
            a.vout[3 * i + c] = vfull;
        else
            a.v[3 * i + c] = vn;
    }
    if (a.peek) return;  // the read-only force pass of velocity-Verlet
    st_rec(Rout + 2 * i, make_float4(ni.x, ni.y, ni.z, H[0]),
           make_float4(H[1], H[2], bf_pack(L[1], L[0]), bf_pack(0.0f, L[2])));
    a.lo32[i] = make_float4(L[0], L[1], L[2], 0.0f);
    const float wi = a.wsum_inv[i];
    a.damage[i] = wi > 0.0f ? fmaxf(0.0f, 1.0f - ws * wi) : 0.0f;
    if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
}

// Both kernels walk the family like the bond-based step: chunks of kUnroll
// slots, ids and records of a chunk requested together, dead slots masked with
// selects; bonds near or past s_c are decided after their flag word.
template <int SCM, bool UW>
__global__ void __launch_bounds__(256) k_osb32_dilation(const __grid_constant__ StepArgsF32 a,
                                                        const OsbArgs32 o)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const int cur = (int)(step & 1);
    const float4* __restrict__ R = a.rec[cur];
    const int64_t W = 32LL * a.Q;
    const int64_t nslices = (a.n + 31) >> 5;
    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int64_t i = (g << 5) + lane;
        const int Wg = a.sw[g];
        const int32_t* __restrict__ col = a.nbr + g * W * 32 + lane;
        float4 ai, bi;
        ld_rec(R + 2 * i, ai, bi);
        const LanePairs pi = lane_pairs(ai, bi);
        const float wc = UW ? lane_wconst(a, i) : 0.0f;
        // per instance in a batch, as in the bond-based step
        const float fast_lo = a.inst != nullptr ? a.itab[a.inst[i]].fast_lo : a.fast_lo;
        uint32_t* bw = a.bits + g * a.Q * 32 + lane;
        float acc = 0.0f;
        uint32_t word = 0u, nword = 0u, pend = 0u;
        const int nch = (Wg + kUnroll - 1) / kUnroll;
        int32_t jn[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) jn[u] = __ldg(col + u * 32);
        for (int c = 0; c < nch; ++c) {
            const int m0 = c * kUnroll;
            const int q = m0 >> 5, b0 = m0 & 31;
            if (b0 == 0) {
                word = bw[q * 32];
                nword = word;
                pend = 0u;
            }
            int32_t jj[kUnroll];
            float4 ra[kUnroll], rb[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) jj[u] = jn[u];
            if (c + 1 < nch) {  // ids of the next chunk while this one is evaluated
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) jn[u] = __ldg(col + (m0 + kUnroll + u) * 32);
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) ld_rec(R + 2 * (int64_t)jj[u], ra[u], rb[u]);
            const uint32_t wb = word >> b0;
            uint32_t pc = 0u;
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const bool alive = (wb >> u) & 1u;
                const BondF32 bd = bond_f32_pk(pi, ra[u], rb[u]);
                const bool cand = bd.num >= fast_lo * bd.den;
                pc |= cand ? (1u << u) : 0u;
                // |xi| e V_j = num |xi|^2 V_j / den, |xi|^2 = |y|^2 - num
                const float contrib =
                    __fdividef(bd.num * (bd.y2 - bd.num), bd.den) * node_w<UW>(a, jj[u], wc);
                acc += (alive && !cand) ? contrib : 0.0f;
            }
            pend |= (pc & wb) << b0;
            if (b0 + kUnroll == 32 || c + 1 == nch) {
                while (pend) {
                    const int b = __ffs(pend) - 1;
                    pend &= pend - 1u;
                    const int64_t slot = (g * W + q * 32 + b) * 32 + lane;
                    const int32_t j = col[(int64_t)(q * 32 + b) * 32];
                    bool brk;
                    resolve_bond<SCM, UW>(a, cur, i, j, slot, &brk);
                    if (brk) {
                        nword &= ~(1u << b);
                    } else {
                        float4 ra1, rb1;
                        ld_rec(R + 2 * (int64_t)j, ra1, rb1);
                        const BondF32 bd = bond_f32_pk(pi, ra1, rb1);
                        acc += __fdividef(bd.num * (bd.y2 - bd.num), bd.den) * node_w<UW>(a, j, wc);
                    }
                }
                if (nword != word) bw[q * 32] = nword;
            }
        }
        const float m = o.mvol[i];
        const float th = m > 0.0f ? 3.0f * acc / m : 0.0f;
        o.theta[i] = th;
        const float be = o.ab[i].y;  // static: set up once from m
        o.ab[i].x = m > 0.0f ? (float)(3.0 * o.K * th / (o.delta * m)) - be * th / 3.0f : 0.0f;
    }
}

template <int SCM, bool UW>
__global__ void __launch_bounds__(256, 3) k_osb32_force(const __grid_constant__ StepArgsF32 a,
                                                     const OsbArgs32 o)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const int cur = (int)(step & 1);
    const float4* __restrict__ R = a.rec[cur];
    float4* __restrict__ Rout = const_cast<float4*>(a.rec[cur ^ 1]);
    const int64_t W = 32LL * a.Q;
    const int64_t nslices = (a.n + 31) >> 5;
    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int64_t i = (g << 5) + lane;
        const int Wg = a.sw[g];
        const int32_t* __restrict__ col = a.nbr + g * W * 32 + lane;
        float4 ai, bi;
        ld_rec(R + 2 * i, ai, bi);
        const NodeF32 ni = unpack(ai, bi);
        const LanePairs pi = lane_pairs(ai, bi);
        const float wc = UW ? lane_wconst(a, i) : 0.0f;
        const float2 abi = o.ab[i];
        const float al = abi.x, be = abi.y;
        const uint32_t* bw = a.bits + g * a.Q * 32 + lane;
        float fx = 0.f, fy = 0.f, fz = 0.f, ws = 0.f;
        uint32_t word = 0u;
        const int nch = (Wg + kUnroll - 1) / kUnroll;
        int32_t jn[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) jn[u] = __ldg(col + u * 32);
        for (int c = 0; c < nch; ++c) {
            const int m0 = c * kUnroll;
            const int q = m0 >> 5, b0 = m0 & 31;
            if (b0 == 0) word = bw[q * 32];
            int32_t jj[kUnroll];
            float4 ra[kUnroll], rb[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) jj[u] = jn[u];
            if (c + 1 < nch) {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) jn[u] = __ldg(col + (m0 + kUnroll + u) * 32);
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) ld_rec(R + 2 * (int64_t)jj[u], ra[u], rb[u]);
            const uint32_t wb = word >> b0;
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const bool alive = (wb >> u) & 1u;
                const BondF32 bd = bond_f32_pk(pi, ra[u], rb[u]);
                const float2 abj = __ldg(o.ab + jj[u]);  // written by the dilation launch
                const float xx = bd.y2 - bd.num;        // |xi|^2
                const float L = xx * rsqrtf(xx);
                const float e = __fdividef(bd.num * L, bd.den);
                const float t = (al + abj.x) * L + (be + abj.y) * e;  // t'_ij + t'_ji
                const float vj = node_w<UW>(a, jj[u], wc);
                float f = t * vj * rsqrtf(bd.y2);
                f = alive ? f : 0.0f;
                fx = fmaf(f, bd.yx, fx);
                fy = fmaf(f, bd.yy, fy);
                fz = fmaf(f, bd.yz, fz);
                ws += alive ? vj : 0.0f;
            }
        }
        if (i < a.n) integrate_osb_f32(a, i, step, fx, fy, fz, ws, ni, Rout);
    }
}

// weighted volume m (horizon units) and beta' of every node
__global__ void k_osb32_setup(const StepArgsF32 a, const OsbArgs32 o)
{
    const int64_t W = 32LL * a.Q;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < (((a.n + 31) >> 5) << 5);
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = p >> 5;
        const int lane = (int)(p & 31);
        double m = 0.0;
        for (int k = 0; k < a.sw[g]; ++k) {
            const int64_t slot = (g * W + k) * 32 + lane;
            const int64_t j = a.nbr[slot];
            double L = 0.0;
            if (j != p) {
                const double e0 = a.x64[3 * j] - a.x64[3 * p], e1 = a.x64[3 * j + 1] - a.x64[3 * p + 1],
                             e2 = a.x64[3 * j + 2] - a.x64[3 * p + 2];
                L = sqrt(e0 * e0 + e1 * e1 + e2 * e2) * a.inv_delta;
            }
            if ((a.bits[(g * a.Q + (k >> 5)) * 32 + lane] >> (k & 31)) & 1u)
                m += L * L * (double)node_w<false>(a, j, 0.0f);
        }
        o.mvol[p] = (float)m;
        o.ab[p] = make_float2(0.0f, m > 0.0 ? (float)(15.0 * o.G / (o.delta * m)) : 0.0f);
    }
}

}  // namespace

cudaError_t launch_osb32_setup(const StepArgsF32& a, const OsbArgs32& o, cudaStream_t s)
{
    int64_t g = ((((a.n + 31) >> 5) << 5) + 255) / 256;
    k_osb32_setup<<<(int)(g < 1 ? 1 : g), 256, 0, s>>>(a, o);
    return cudaGetLastError();
}

namespace {
template <int SCM, bool UW>
cudaError_t osb32_step(const StepArgsF32& a, const OsbArgs32& o, int grid, int grid_dil,
                       int block, cudaStream_t s)
{
    k_osb32_dilation<SCM, UW><<<grid_dil, block, 0, s>>>(a, o);
    if (cudaPeekAtLastError() == cudaSuccess) k_osb32_force<SCM, UW><<<grid, block, 0, s>>>(a, o);
    return cudaGetLastError();
}
}  // namespace

const void* osb32_dilation_kernel(int sc_mode, bool uniform_w)
{
    if (sc_mode == 0)
        return uniform_w ? (const void*)k_osb32_dilation<0, true> : (const void*)k_osb32_dilation<0, false>;
    return uniform_w ? (const void*)k_osb32_dilation<1, true> : (const void*)k_osb32_dilation<1, false>;
}

const void* osb32_force_kernel(int sc_mode, bool uniform_w)
{
    if (sc_mode == 0)
        return uniform_w ? (const void*)k_osb32_force<0, true> : (const void*)k_osb32_force<0, false>;
    return uniform_w ? (const void*)k_osb32_force<1, true> : (const void*)k_osb32_force<1, false>;
}

cudaError_t launch_osb32_step(const StepArgsF32& a, const OsbArgs32& o, int sc_mode, int grid,
                              int grid_dil, int block, cudaStream_t s)
{
    if (sc_mode == 0)
        return a.uniform_w ? osb32_step<0, true>(a, o, grid, grid_dil, block, s)
                           : osb32_step<0, false>(a, o, grid, grid_dil, block, s);
    return a.uniform_w ? osb32_step<1, true>(a, o, grid, grid_dil, block, s)
                       : osb32_step<1, false>(a, o, grid, grid_dil, block, s);
}
}  // namespace pd
