// Ordinary state-based linear solid (constant influence function) in
// double-word FP32 arithmetic, for PD_PREC_DW handles with model 1: the two
// loops of k_osb_dilation / k_osb_force (pd_step_osb.cu) on the double-word
// records, lengths and node-state layout of the double-word bond-based step
// (pd_step_dw.cu).
//
// In units of the horizon delta (L~ = |xi| / delta, e~ = e / delta) the
// model's terms are
//   m~_i    = sum_j |xi~|^2 V_j                            (m = delta^2 m~, once)
//   theta_i = 3 sum_j mu_ij L~ e~ V_j / m~_i                (dimensionless)
//   alpha~_i = 3 K theta_i / m~_i - beta~_i theta_i / 3,  beta~_i = 15 G / m~_i
//   F_i     = (1 / delta) sum_j mu_ij [(alpha~_i + alpha~_j) L~ + (beta~_i + beta~_j) e~] V_j y / |y|
// and e~ = s L~ with the stretch s of the bond-based double-word step
// (cancellation-free, exact leading position differences).  Bonds break in
// the dilation loop (Eq. 6), decided against the FP64 s_c for stretches in
// the band below the smallest s_c; the force loop reads the flags it left.
// Per node the coefficients alpha~, beta~ are published as double-words
// ({alpha_h, alpha_l, beta_h, beta_l}, one 128-bit load per neighbour); the
// integration (Euler-Cromer or velocity-Verlet), boundary conditions and
// damage are the bond-based double-word step's, in FP64.
#include <cuda_runtime.h>

#include "pd_dw.h"
#include "pd_internal.h"

namespace pd {
namespace {

using namespace dwa;

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

__device__ __forceinline__ void split(double x, float& h, float& l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

// stretch, deformed bond vector and 1/|y| of one bond (the bond-based
// double-word step's arithmetic)
struct OsbBondDw {
    Dw s, ir;
    Dw y[3];
};

__device__ __forceinline__ OsbBondDw osb_bond_dw(const OwnDw& o, const Rec& j, const float2 len)
{
    const float jxh[3] = {j.a0.x, j.a0.y, j.a0.z}, juh[3] = {j.a0.w, j.a1.x, j.a1.y};
    const float jxl[3] = {j.b0.x, j.b0.y, j.b0.z}, jul[3] = {j.b0.w, j.b1.x, j.b1.y};
    OsbBondDw out;
    Dw nm[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const Dw xi{jxh[c] - o.xh[c], jxl[c] - o.xl[c]};  // exact leading difference
        Dw et = two_sum(juh[c], -o.uh[c]);
        et.l += jul[c] - o.ul[c];
        out.y[c] = dw_add(xi, et);
        nm[c] = dw_mul(et, dw_add(xi, out.y[c]));
    }
    Dw num = two_sum(nm[0].h, nm[1].h);
    num.l += nm[0].l + nm[1].l;
    num = dw_add(num, nm[2]);
    const Dw L{len.x, len.y};
    Dw r;
    dw_norm(dw_add(dw_mul(L, L), num), r, out.ir);
    out.s = dw_div(num, dw_mul(L, dw_add(L, r)));
    return out;
}

// m~_i and beta~_i once (bond flags after the initial cuts), in FP64
__global__ void k_osb_dw_setup(const StepArgsF64 a, OsbDwArgs o)
{
    const int64_t W = 32LL * a.Q;
    const int64_t total = ((a.n + 31) >> 5) << 5;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = p >> 5;
        const int lane = (int)(p & 31);
        double acc = 0.0;
        for (int m = 0; m < a.sw[g]; ++m) {
            if (!((a.bits[(g * a.Q + (m >> 5)) * 32 + lane] >> (m & 31)) & 1u)) continue;
            const int64_t slot = (g * W + m) * 32 + lane;
            const float2 len = o.len[slot];
            const double L = (double)len.x + (double)len.y;
            acc += L * L * o.vol[a.nbr[slot]];
        }
        o.mvol[p] = acc;
        const double be = acc > 0.0 ? 15.0 * o.G / acc : 0.0;
        float bh, bl;
        split(be, bh, bl);
        o.ab[p] = make_float4(0.0f, 0.0f, bh, bl);
    }
}

// A bond whose leading stretch word reached the band below the smallest s_c:
// decided in FP64 (recomputed with the same arithmetic), then the no-fail rule.
__device__ __noinline__ OsbBondDw osb_resolve_dw(const StepArgsF64& a, const float4* R, int64_t i,
                                                 int64_t j, float2 len, bool* broken)
{
    Rec own, nb;
    ld_rec(R + 4 * i, own.a0, own.a1);
    ld_rec(R + 4 * i + 2, own.b0, own.b1);
    ld_rec(R + 4 * j, nb.a0, nb.a1);
    ld_rec(R + 4 * j + 2, nb.b0, nb.b1);
    const OsbBondDw bd = osb_bond_dw(own_of(own), nb, len);
    bool brk = (double)bd.s.h + (double)bd.s.l >= bond_sc(a, i, j);
    if (brk && a.has_nofail) brk = ((a.bct[a.bcc[i]].mask | a.bct[a.bcc[j]].mask) & 8u) == 0u;
    *broken = brk;
    return bd;
}

__global__ void __launch_bounds__(256, 2)
    k_osb_dw_dilation(const __grid_constant__ StepArgsF64 a, const __grid_constant__ DwArgs d,
                      const __grid_constant__ OsbDwArgs o)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const float4* __restrict__ R = d.rec[step & 1];
    const int Q = a.Q;
    const int64_t W = 32LL * Q;
    const int64_t nslices = (a.n + 31) >> 5;
    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int Wg = a.sw[g];
        const int32_t* __restrict__ col = a.nbr + g * W * 32 + lane;
        const int64_t i = (g << 5) + lane;
        Rec me;
        ld_rec(R + 4 * i, me.a0, me.a1);
        ld_rec(R + 4 * i + 2, me.b0, me.b1);
        const OwnDw own = own_of(me);
        uint32_t* bw = a.bits + g * Q * 32 + lane;
        // band below the smallest s_c the node's bonds can have (per instance in
        // a batch: both ends of a bond belong to the same instance)
        const float fast_lo = a.inst != nullptr
                                  ? (float)((1.0 - 0x1.0p-20) * a.itab[a.inst[i]].sc_lo)
                                  : d.fast_lo;
        Dw acc{0.f, 0.f};  // sum of L~ e~ V_j over intact bonds
        const int nch = (Wg + 1) >> 1;
        int32_t jn0 = __ldg(col), jn1 = __ldg(col + 32);
        uint32_t word = 0u, nword = 0u, pend = 0u;
        for (int c = 0; c < nch; ++c) {
            const int m0 = 2 * c;
            const int q = m0 >> 5, b0 = m0 & 31;
            if (b0 == 0) {
                word = bw[q * 32];
                nword = word;
                pend = 0u;
            }
            const int32_t jj[2] = {jn0, jn1};
            if (c + 1 < nch) {
                jn0 = __ldg(col + (m0 + 2) * 32);
                jn1 = __ldg(col + (m0 + 3) * 32);
            }
            const uint32_t wb = word >> b0;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                Rec nb;
                ld_rec(R + 4 * (int64_t)jj[u], nb.a0, nb.a1);
                ld_rec(R + 4 * (int64_t)jj[u] + 2, nb.b0, nb.b1);
                const float2 len = __ldg(d.len + (g * W + m0 + u) * 32 + lane);
                const OsbBondDw bd = osb_bond_dw(own, nb, len);
                const bool cand = bd.s.h >= fast_lo;
                const bool ok = ((wb >> u) & 1u) && !cand;
                pend |= (cand && ((wb >> u) & 1u) ? 1u : 0u) << (b0 + u);
                const Dw L{len.x, len.y};
                const Dw t = dw_mul(dw_mul(bd.s, dw_mul(L, L)), Dw{nb.a1.z, nb.a1.w});
                const Dw sum = two_sum(acc.h, ok ? t.h : 0.0f);
                acc.h = sum.h;
                acc.l += sum.l + (ok ? t.l : 0.0f);
            }
            if (b0 + 2 == 32 || c + 1 == nch) {  // end of bond-flag word q
                while (pend) {
                    const int b = __ffs(pend) - 1;
                    pend &= pend - 1u;
                    const int64_t slot = (g * W + q * 32 + b) * 32 + lane;
                    const int64_t j = col[(int64_t)(q * 32 + b) * 32];
                    const float2 len = d.len[slot];
                    bool broken;
                    const OsbBondDw bd = osb_resolve_dw(a, R, i, j, len, &broken);
                    if (broken) {
                        nword &= ~(1u << b);
                    } else {
                        float4 c0, c1;
                        ld_rec(R + 4 * j, c0, c1);
                        const Dw L{len.x, len.y};
                        const Dw t = dw_mul(dw_mul(bd.s, dw_mul(L, L)), Dw{c1.z, c1.w});
                        const Dw sum = two_sum(acc.h, t.h);
                        acc.h = sum.h;
                        acc.l += sum.l + t.l;
                    }
                }
                if (nword != word) bw[q * 32] = nword;
            }
        }
        if (i < a.n) {
            const double m = o.mvol[i];
            const double th = m > 0.0 ? 3.0 * ((double)acc.h + (double)acc.l) / m : 0.0;
            const float4 ab = o.ab[i];
            const double be = (double)ab.z + (double)ab.w;
            const double al = m > 0.0 ? 3.0 * o.K * th / m - be * th / 3.0 : 0.0;
            float ah, alo;
            split(al, ah, alo);
            o.theta[i] = th;
            o.ab[i] = make_float4(ah, alo, ab.z, ab.w);
        }
    }
}

template <bool UW>
__global__ void __launch_bounds__(256, 2)
    k_osb_dw_force(const __grid_constant__ StepArgsF64 a, const __grid_constant__ DwArgs d,
                   const __grid_constant__ OsbDwArgs o)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const int cur = (int)(step & 1);
    const float4* __restrict__ R = d.rec[cur];
    float4* __restrict__ Rout = const_cast<float4*>(d.rec[cur ^ 1]);
    const double2* __restrict__ rin = reinterpret_cast<const double2*>(a.rec[cur]);
    double2* __restrict__ rout = reinterpret_cast<double2*>(const_cast<double*>(a.rec[cur ^ 1]));
    const int Q = a.Q;
    const int64_t W = 32LL * Q;
    const int64_t nslices = (a.n + 31) >> 5;
    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int Wg = a.sw[g];
        const int32_t* __restrict__ col = a.nbr + g * W * 32 + lane;
        const int64_t i = (g << 5) + lane;
        Rec me;
        ld_rec(R + 4 * i, me.a0, me.a1);
        ld_rec(R + 4 * i + 2, me.b0, me.b1);
        const OwnDw own = own_of(me);
        const float4 abi = o.ab[i];
        const Dw ai{abi.x, abi.y}, bi{abi.z, abi.w};
        Dw F[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        Dw ws{0.f, 0.f};
        int alive_count = 0;
        const int nch = (Wg + 1) >> 1;
        int32_t jn0 = __ldg(col), jn1 = __ldg(col + 32);
        uint32_t word = 0u;
        for (int c = 0; c < nch; ++c) {
            const int m0 = 2 * c;
            const int q = m0 >> 5, b0 = m0 & 31;
            if (b0 == 0) {
                word = a.bits[(g * Q + q) * 32 + lane];
                alive_count += __popc(word);
            }
            const int32_t jj[2] = {jn0, jn1};
            if (c + 1 < nch) {
                jn0 = __ldg(col + (m0 + 2) * 32);
                jn1 = __ldg(col + (m0 + 3) * 32);
            }
            const uint32_t wb = word >> b0;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                Rec nb;
                ld_rec(R + 4 * (int64_t)jj[u], nb.a0, nb.a1);
                ld_rec(R + 4 * (int64_t)jj[u] + 2, nb.b0, nb.b1);
                const float4 abj = __ldg(o.ab + jj[u]);
                const float2 len = __ldg(d.len + (g * W + m0 + u) * 32 + lane);
                const OsbBondDw bd = osb_bond_dw(own, nb, len);
                const Dw L{len.x, len.y};
                // (t_ij + t_ji) delta = (alpha~_i + alpha~_j) L~ + (beta~_i + beta~_j) e~
                const Dw t = dw_add(dw_mul(dw_add(ai, Dw{abj.x, abj.y}), L),
                                    dw_mul(dw_add(bi, Dw{abj.z, abj.w}), dw_mul(bd.s, L)));
                const Dw Vj{nb.a1.z, nb.a1.w};
                Dw coef = dw_mul(dw_mul(t, Vj), bd.ir);
                const bool ok = (wb >> u) & 1u;
                coef = Dw{ok ? coef.h : 0.0f, ok ? coef.l : 0.0f};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const Dw f = dw_mul(coef, bd.y[k]);
                    const Dw sum = two_sum(F[k].h, f.h);
                    F[k].h = sum.h;
                    F[k].l += sum.l + f.l;
                }
                if (!UW) {
                    const Dw sum = two_sum(ws.h, ok ? Vj.h : 0.0f);
                    ws.h = sum.h;
                    ws.l += sum.l + (ok ? Vj.l : 0.0f);
                }
            }
        }
        if (i >= a.n) continue;
        // damped Euler-Cromer update, boundary conditions and damage (as the
        // bond-based double-word step)
        const uint32_t cls = a.bcc[i];
        uint32_t mask = 0u;
        double gdisp[3] = {0.0, 0.0, 0.0};
        double Fn[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) Fn[k] = ((double)F[k].h + (double)F[k].l) * d.inv_delta;
        if (cls != 0u) {
            const BcClass& bc = a.bct[cls];
            mask = bc.mask;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gdisp[k] = bc.disp[k];
                Fn[k] += a.load * bc.force[k];
            }
        }
        const double s_now = bc_scale(a.disp_rate, a.ramp_steps, step);
        const double s_next = bc_scale(a.disp_rate, a.ramp_steps, step + 1);
        const double2 u01 = rin[4 * i + 2], u23 = rin[4 * i + 3];
        const double uo[3] = {u01.x, u01.y, u23.x};
        const bool first = a.vv && step == a.step_ctr[1];
        double un[3];
        float uh[3], ul[3];
        bool finite = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double vi = a.v[3 * i + k];
            const double adt = (Fn[k] - a.eta * vi) * d.dt_rho;  // dt a
            double vn, vfull;
            if (a.vv) {
                vfull = first ? vi : vi + 0.5 * adt;
                vn = vfull + 0.5 * adt;
            } else {
                vn = vi + adt;
                vfull = vn;
            }
            double u = uo[k] + a.dt * vn;
            if (mask & (1u << k)) {
                u = gdisp[k] * s_next;
                vn = gdisp[k] * (s_next - s_now) / a.dt;
                vfull = vi;
            }
            finite = finite && isfinite(u);
            un[k] = u;
            if (a.peek)
                a.vout[3 * i + k] = vfull;
            else
                a.v[3 * i + k] = vn;
            split(u * d.inv_delta, uh[k], ul[k]);
        }
        if (a.peek) continue;  // the read-only force pass of velocity-Verlet
        rout[4 * i] = rin[4 * i];
        rout[4 * i + 1] = rin[4 * i + 1];
        rout[4 * i + 2] = make_double2(un[0], un[1]);
        rout[4 * i + 3] = make_double2(un[2], 0.0);
        st_rec(Rout + 4 * i, make_float4(me.a0.x, me.a0.y, me.a0.z, uh[0]),
               make_float4(uh[1], uh[2], me.a1.z, me.a1.w));
        st_rec(Rout + 4 * i + 2, make_float4(me.b0.x, me.b0.y, me.b0.z, ul[0]),
               make_float4(ul[1], ul[2], 0.0f, 0.0f));
        const double wsum = UW ? d.w_const * (double)alive_count : (double)ws.h + (double)ws.l;
        const double wi = a.wsum_inv[i];
        a.damage[i] = wi > 0.0 ? fmax(0.0, 1.0 - wsum * wi) : 0.0;
        if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
    }
}

int grid_nodes(int64_t n)
{
    const int64_t b = ((((n + 31) >> 5) << 5) + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace

cudaError_t launch_osb_dw_setup(const StepArgsF64& a, const OsbDwArgs& o, cudaStream_t s)
{
    k_osb_dw_setup<<<grid_nodes(a.n), 256, 0, s>>>(a, o);
    return cudaGetLastError();
}

cudaError_t launch_osb_dw_step(const StepArgsF64& a, const DwArgs& d, const OsbDwArgs& o, int grid,
                               int block, cudaStream_t s)
{
    k_osb_dw_dilation<<<grid, block, 0, s>>>(a, d, o);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (d.uniform_w)
        k_osb_dw_force<true><<<grid, block, 0, s>>>(a, d, o);
    else
        k_osb_dw_force<false><<<grid, block, 0, s>>>(a, d, o);
    return cudaGetLastError();
}

}  // namespace pd
