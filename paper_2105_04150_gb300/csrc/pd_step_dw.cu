// FP64-grade peridynamic step from double-word FP32 arithmetic (sm_103a).
//
// GB300 issues FP32 operations at about 58 times its FP64 rate, and the FP64
// step kernel is bound by the FP64 pipe.  This kernel computes the same step
// (Eq. 4 stretch, Eq. 6 breaking, Eq. 5/10 force, Eq. 11 update, Eq. 8
// damage) with every bond quantity carried as an unevaluated sum of two FP32
// numbers (double-word arithmetic, pd_dw.h), about 48 significant bits: the
// relative accuracy of a bond force is ~1e-13, far inside the FP64 parity bar,
// for about two hundred FP32 operations instead of ~30 FP64 ones.  Variants:
// sc_mode, uniform or per-node weights (batches take the latter), softening
// (the stored FP64 integrity scales the force; bonds near s_0 are resolved in
// FP64), per-bond stiffness (a run-time branch), velocity-Verlet (its own
// translation unit, below).
//
// Work decomposition, bond flags, node order and the double-buffered records
// are those of the FP32 kernel (lane per node over the sliced family).
// Node state stays FP64: each node's owner keeps u and v in the FP64 records
// and integrates in FP64; what neighbours read is a 64-byte double-word copy
//   {xh.x, xh.y, xh.z, uh.x} {uh.y, uh.z, wh, wl} {xl.x, xl.y, xl.z, ul.x} {ul.y, ul.z, 0, 0}
// with positions x~ = (x - origin) / delta and u~ = u / delta in units of the
// horizon and w = c V, read as two 256-bit loads.  The origin puts every
// position component at least B horizons above zero, B above the largest
// component of any bond, so the leading words of two bonded positions are
// within a factor 2 and their difference is exact (Sterbenz's lemma).  The
// reference length |xi| / delta of each slot is a double-word computed once
// in FP64.
//
// Per bond, with xi and eta the double-word differences (exact leading
// parts): y = xi + eta, num = eta . (2 xi + eta) = |y|^2 - |xi|^2 without
// cancellation, |y|^2 = L^2 + num, s = num / (L (L + |y|)), and the force
// c V s y / |y|.  |y|, 1/|y| and the quotient come from FP32 seeds
// (approximate rsqrt / rcp, one Newton step) with a double-word correction.
// Both directions of a bond produce the same s bit for bit (every operation
// is odd or even under exchanging i and j), so they break together.  A bond
// whose leading stretch word reaches a band just below the smallest s_c is
// decided at the end of its flag word against the FP64 s_c, as in the FP32
// kernel; the rest of the break test needs no FP64 operation.
#include <cuda_runtime.h>

#include "pd_dw.h"
#include "pd_internal.h"

namespace pd {
namespace {

#ifndef PD_DW_MIN_BLOCKS
#define PD_DW_MIN_BLOCKS 2
#endif
#ifndef PD_DW_PREFETCH
#define PD_DW_PREFETCH 1
#endif
// Velocity-Verlet build (pd_step_dw_vv.cu includes this file with PD_DW_VV 1):
// the velocity-Verlet epilogue and the read-only force pass, compiled apart from
// the Euler-Cromer one so that the latter's bond loop keeps its code.  A
// separate translation unit, not a template parameter: ptxas 13.0.88 fails on
// this kernel with a fourth one.
#ifndef PD_DW_VV
#define PD_DW_VV 0
#endif
constexpr bool VV = PD_DW_VV != 0;

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

using namespace dwa;

struct BondDw {
    Dw s;     // stretch
    Dw coef;  // s / |y| (times w_j unless the weights are uniform)
    Dw y[3];  // deformed bond vector / delta
};

// One bond of the lane's node.  `len` is the slot's |xi| / delta (slots
// without a bond hold 1 and their neighbour is the node itself).
template <bool UW>
__device__ __forceinline__ BondDw bond_dw(const OwnDw& o, const Rec& j, const float2 len)
{
    const float jxh[3] = {j.a0.x, j.a0.y, j.a0.z}, juh[3] = {j.a0.w, j.a1.x, j.a1.y};
    const float jxl[3] = {j.b0.x, j.b0.y, j.b0.z}, jul[3] = {j.b0.w, j.b1.x, j.b1.y};
    BondDw out;
    Dw nm[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        // xi = x_j - x_i and eta = u_j - u_i, the leading differences exact: for
        // positions by construction of their origin (Sterbenz), for
        // displacements by a two-sum
        const Dw xi{jxh[c] - o.xh[c], jxl[c] - o.xl[c]};
        Dw et = two_sum(juh[c], -o.uh[c]);
        et.l += jul[c] - o.ul[c];
        out.y[c] = dw_add(xi, et);
        nm[c] = dw_mul(et, dw_add(xi, out.y[c]));  // eta_c (2 xi_c + eta_c)
    }
    // num = eta . (2 xi + eta) = |y|^2 - |xi|^2
    Dw num = two_sum(nm[0].h, nm[1].h);
    num.l += nm[0].l + nm[1].l;
    num = dw_add(num, nm[2]);
    const Dw L{len.x, len.y};
    const Dw y2 = dw_add(dw_mul(L, L), num);
    Dw r, ir;
    dw_norm(y2, r, ir);
    // s = num / den, den = L (L + |y|): FP32 quotient plus the remainder's
    out.s = dw_div(num, dw_mul(L, dw_add(L, r)));
    out.coef = dw_mul(out.s, ir);
    if (!UW) out.coef = dw_mul(out.coef, Dw{j.a1.z, j.a1.w});
    return out;
}

// per-bond stiffness c_ij (a double-word per slot) on the coefficient
__device__ __forceinline__ void scale_coef(BondDw& b, const float2 c)
{
    b.coef = dw_mul(b.coef, Dw{c.x, c.y});
}

// F += coef y when `ok` (a select: whatever a masked slot computed, including
// a non-finite value, is dropped)
__device__ __forceinline__ void add_force(Dw (&F)[3], const BondDw& b, bool ok)
{
    const Dw cf{ok ? b.coef.h : 0.0f, ok ? b.coef.l : 0.0f};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const Dw f = dw_mul(cf, b.y[k]);
        const Dw t = two_sum(F[k].h, f.h);
        F[k].h = t.h;
        F[k].l += t.l + f.l;
    }
}

// A bond whose leading stretch word reached the band below the smallest s_c:
// recomputed with the same arithmetic and decided in FP64 against its s_c,
// then the no-fail rule.
template <int SCM, bool UW, bool SOFT>
__device__ __noinline__ BondDw resolve_dw(const StepArgsF64& a, const DwArgs& d, int cur,
                                          int64_t i, int64_t j, int64_t slot, bool* broken,
                                          double* mu_out)
{
    const float4* __restrict__ R = d.rec[cur];
    Rec own, nb;
    ld_rec(R + 4 * i, own.a0, own.a1);
    ld_rec(R + 4 * i + 2, own.b0, own.b1);
    ld_rec(R + 4 * j, nb.a0, nb.a1);
    ld_rec(R + 4 * j + 2, nb.b0, nb.b1);
    BondDw bd = bond_dw<UW>(own_of(own), nb, d.len[slot]);
    if (d.cb != nullptr) scale_coef(bd, d.cb[slot]);
    double sc = a.sc;
    if (a.inst != nullptr) {  // batch: the instance's own parameters, local ids as keys
        const InstParams& ip = a.itab[a.inst[i]];
        sc = ip.sc_mode == 1 ? sc_draw(ip.sc_seed, ip.sc_lo, ip.sc_hi, a.hid[i], a.hid[j]) : ip.sc;
    } else if (SCM == 1) {
        sc = sc_draw(a.sc_seed, a.sc_lo, a.sc_hi, a.gid[i], a.gid[j]);
    }
    const double s64 = (double)bd.s.h + (double)bd.s.l;
    bool brk = s64 >= sc;
    if (brk && a.has_nofail) brk = ((a.bct[a.bcc[i]].mask | a.bct[a.bcc[j]].mask) & 8u) == 0u;
    *broken = brk;
    double mu = 1.0;
    if (SOFT) {
        // the integrity only decreases, as the stretch passes s_0 = s_c / kr (a
        // no-fail bond past s_c keeps 0); the force is scaled by it
        if (brk) {
            a.integ[slot] = 0.0;
        } else {
            mu = a.integ[slot];
            const double s0 = sc / a.kr;
            if (s64 > s0) {
                const double ms = s64 >= sc ? 0.0 : soft_mu_of(s64, s0, sc, a.k1, a.beta);
                if (ms < mu) {
                    mu = ms;
                    a.integ[slot] = ms;
                }
            }
            const float mh = (float)mu;
            bd.coef = dw_mul(bd.coef, Dw{mh, (float)(mu - (double)mh)});
        }
    }
    *mu_out = mu;
    return bd;
}

// softening: a bond's stored integrity scales its force (the fast path needs no
// FP64 operation for the unsoftened ones, recognised by their bit pattern);
// returns mu - 1 for the damage weight
__device__ __forceinline__ double soften(BondDw& b, const double* integ, int64_t slot)
{
    const unsigned long long bits = __ldg(reinterpret_cast<const unsigned long long*>(integ) + slot);
    if (bits == 0x3FF0000000000000ull) return 0.0;  // mu = 1
    const double mu = __longlong_as_double(bits);
    const float mh = (float)mu;
    b.coef = dw_mul(b.coef, Dw{mh, (float)(mu - (double)mh)});
    return mu - 1.0;
}

template <int SCM, bool UW, bool SOFT>
__global__ void __launch_bounds__(256, PD_DW_MIN_BLOCKS)
    k_step_dw(const __grid_constant__ StepArgsF64 a, const __grid_constant__ DwArgs d)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const int cur = (int)(step & 1);
    const int Q = a.Q;
    const int64_t W = 32LL * Q;
    const int64_t nslices = (a.n + 31) >> 5;
    const float4* __restrict__ R = d.rec[cur];
    float4* __restrict__ Rout = const_cast<float4*>(d.rec[cur ^ 1]);
    const double2* __restrict__ rin = reinterpret_cast<const double2*>(a.rec[cur]);
    double2* __restrict__ rout = reinterpret_cast<double2*>(const_cast<double*>(a.rec[cur ^ 1]));

    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int Wg = a.sw[g];
        const int32_t* __restrict__ col = a.nbr + g * W * 32 + lane;
        if (lane == 0) prefetch_l2(col, (uint32_t)(((Wg + 3) & ~3) * 128));
        const int64_t i = (g << 5) + lane;
        Rec me;
        ld_rec(R + 4 * i, me.a0, me.a1);
        ld_rec(R + 4 * i + 2, me.b0, me.b1);
        const OwnDw own = own_of(me);
        uint32_t* bw = a.bits + g * Q * 32 + lane;
        // band below the smallest s_c the node's bonds can have (per instance in a
        // batch: both ends of a bond belong to the same instance)
        const float fast_lo = a.inst != nullptr
                                  ? (float)((1.0 - 0x1.0p-20) * a.itab[a.inst[i]].sc_lo /
                                            (SOFT ? a.kr : 1.0))
                                  : d.fast_lo;
        // force sums of the A and B halves, and (non-uniform weights) the sum of
        // w_j over intact bonds
        Dw F[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        Dw ws{0.f, 0.f};
        int alive_count = 0;
        double wsoft = 0.0;  // softening: sum of (mu - 1) w~_j over intact softened bonds

        // chunks of two slots (bonds A and B); ids one chunk ahead
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
            const int32_t j0 = jn0, j1 = jn1;
            if (c + 1 < nch) {
                jn0 = __ldg(col + (m0 + 2) * 32);
                jn1 = __ldg(col + (m0 + 3) * 32);
            }

            Rec A, B;
            ld_rec(R + 4 * (int64_t)j0, A.a0, A.a1);
            ld_rec(R + 4 * (int64_t)j0 + 2, A.b0, A.b1);
            ld_rec(R + 4 * (int64_t)j1, B.a0, B.a1);
            ld_rec(R + 4 * (int64_t)j1 + 2, B.b0, B.b1);
            const float2 lA = __ldg(d.len + (g * W + m0) * 32 + lane);
            const float2 lB = __ldg(d.len + (g * W + m0 + 1) * 32 + lane);
            const uint32_t wb = word >> b0;
            BondDw bA = bond_dw<UW>(own, A, lA);
            BondDw bB = bond_dw<UW>(own, B, lB);
            if (d.cb != nullptr) {  // per-bond stiffness (a uniform branch)
                scale_coef(bA, __ldg(d.cb + (g * W + m0) * 32 + lane));
                scale_coef(bB, __ldg(d.cb + (g * W + m0 + 1) * 32 + lane));
            }
            const bool candA = bA.s.h >= fast_lo, candB = bB.s.h >= fast_lo;
            const bool okA = (wb & 1u) && !candA, okB = ((wb >> 1) & 1u) && !candB;
            if (SOFT) {
                const double dA = soften(bA, a.integ, (g * W + m0) * 32 + lane);
                const double dB = soften(bB, a.integ, (g * W + m0 + 1) * 32 + lane);
                if (okA && dA != 0.0)
                    wsoft += dA * (UW ? 1.0 : (double)A.a1.z + (double)A.a1.w);
                if (okB && dB != 0.0)
                    wsoft += dB * (UW ? 1.0 : (double)B.a1.z + (double)B.a1.w);
            }
            pend |= (((candA ? 1u : 0u) | (candB ? 2u : 0u)) & wb) << b0;
#if PD_DW_PREFETCH
            // the next chunk's records start toward L1 (their ids have arrived by now)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(R + 4 * (int64_t)jn0));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(R + 4 * (int64_t)jn1));
#endif
            add_force(F, bA, okA);
            add_force(F, bB, okB);
            if (!UW) {
                Dw t = two_sum(ws.h, okA ? A.a1.z : 0.0f);
                ws.h = t.h;
                ws.l += t.l + (okA ? A.a1.w : 0.0f);
                t = two_sum(ws.h, okB ? B.a1.z : 0.0f);
                ws.h = t.h;
                ws.l += t.l + (okB ? B.a1.w : 0.0f);
            }
            if (b0 + 2 == 32 || c + 1 == nch) {  // end of bond-flag word q
                while (pend) {
                    const int b = __ffs(pend) - 1;
                    pend &= pend - 1u;
                    const int64_t slot = (g * W + q * 32 + b) * 32 + lane;
                    const int64_t j = col[(int64_t)(q * 32 + b) * 32];
                    bool broken;
                    double mu;
                    const BondDw f = resolve_dw<SCM, UW, SOFT>(a, d, cur, i, j, slot, &broken, &mu);
                    if (broken) {
                        nword &= ~(1u << b);
                    } else {
                        add_force(F, f, true);
                        float4 c0, c1;
                        if (!UW || (SOFT && mu != 1.0)) ld_rec(R + 4 * j, c0, c1);
                        if (!UW) {
                            const Dw t = two_sum(ws.h, c1.z);
                            ws.h = t.h;
                            ws.l += t.l + c1.w;
                        }
                        if (SOFT && mu != 1.0)
                            wsoft += (mu - 1.0) * (UW ? 1.0 : (double)c1.z + (double)c1.w);
                    }
                }
                if (nword != word) bw[q * 32] = nword;
                alive_count += __popc(nword);
            }
        }

        // ---- integration of the lane's node in FP64 (damped Euler-Cromer, Eq. 11)
        if (i < a.n) {
            const uint32_t cls = a.bcc[i];
            uint32_t mask = 0u;
            double gdisp[3] = {0.0, 0.0, 0.0};
            const double wscale = UW ? d.w_const : 1.0;
            double Fn[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) Fn[k] = ((double)F[k].h + (double)F[k].l) * wscale;
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
            // velocity-Verlet: a^n is formed afresh at the step the state was set
            const bool first = VV && a.vv && step == a.step_ctr[1];
            double un[3];
            float uh[3], ul[3];
            bool finite = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                // stored velocity: v^n (Euler-Cromer) or, for velocity-Verlet, the
                // half-step velocity v^{n-1} + dt/2 a^{n-1} (v^n right after a set state)
                const double vi = a.v[3 * i + k];
                const double adt = (Fn[k] - a.eta * vi) * d.dt_rho;  // dt a
                double vn, vfull;
                if (VV && a.vv) {
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
                if (VV && a.peek)
                    a.vout[3 * i + k] = vfull;
                else
                    a.v[3 * i + k] = vn;
                const double ut = u * d.inv_delta;
                uh[k] = (float)ut;
                ul[k] = (float)(ut - (double)uh[k]);
            }
            if (VV && a.peek) continue;  // the read-only force pass of velocity-Verlet
            rout[4 * i] = rin[4 * i];
            rout[4 * i + 1] = rin[4 * i + 1];
            rout[4 * i + 2] = make_double2(un[0], un[1]);
            rout[4 * i + 3] = make_double2(un[2], 0.0);
            st_rec(Rout + 4 * i, make_float4(me.a0.x, me.a0.y, me.a0.z, uh[0]),
                   make_float4(uh[1], uh[2], me.a1.z, me.a1.w));
            st_rec(Rout + 4 * i + 2, make_float4(me.b0.x, me.b0.y, me.b0.z, ul[0]),
                   make_float4(ul[1], ul[2], 0.0f, 0.0f));
            const double wsum = UW ? d.w_const * ((double)alive_count + wsoft)
                                   : ((double)ws.h + (double)ws.l) + wsoft;
            const double wi = a.wsum_inv[i];
            a.damage[i] = wi > 0.0 ? fmax(0.0, 1.0 - wsum * wi) : 0.0;
            if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
        }
    }
}

// Double-word records of every node from the FP64 records (after a state or
// the weights were set), and the double-word reference length of every slot.
__global__ void k_dw_publish(const double* __restrict__ rec64, float4* __restrict__ rec,
                             int64_t n_pad, double ox, double oy, double oz, double inv_delta)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double* r = rec64 + 8 * p;
        const double xt[3] = {(r[0] - ox) * inv_delta, (r[1] - oy) * inv_delta,
                              (r[2] - oz) * inv_delta};
        const double ut[3] = {r[4] * inv_delta, r[5] * inv_delta, r[6] * inv_delta};
        float xh[3], xl[3], uh[3], ul[3];
        for (int k = 0; k < 3; ++k) {
            xh[k] = (float)xt[k];
            xl[k] = (float)(xt[k] - (double)xh[k]);
            uh[k] = (float)ut[k];
            ul[k] = (float)(ut[k] - (double)uh[k]);
        }
        const float wh = (float)r[3];
        const float wl = (float)(r[3] - (double)wh);
        rec[4 * p] = make_float4(xh[0], xh[1], xh[2], uh[0]);
        rec[4 * p + 1] = make_float4(uh[1], uh[2], wh, wl);
        rec[4 * p + 2] = make_float4(xl[0], xl[1], xl[2], ul[0]);
        rec[4 * p + 3] = make_float4(ul[1], ul[2], 0.0f, 0.0f);
    }
}

__global__ void k_dw_len(const double* __restrict__ x64, const int32_t* __restrict__ nbr,
                         int64_t n, int Q, double inv_delta, float2* __restrict__ len)
{
    const int64_t W = 32LL * Q;
    const int64_t total = ((n + 31) >> 5) << 5;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = p >> 5;
        const int lane = (int)(p & 31);
        for (int m = 0; m < W; ++m) {
            const int64_t slot = (g * W + m) * 32 + lane;
            const int64_t j = nbr[slot];
            float2 v = make_float2(1.0f, 0.0f);  // no bond: a finite placeholder
            if (j != p) {
                const double ex = x64[3 * j] - x64[3 * p], ey = x64[3 * j + 1] - x64[3 * p + 1],
                             ez = x64[3 * j + 2] - x64[3 * p + 2];
                const double L = sqrt(ex * ex + ey * ey + ez * ez) * inv_delta;
                v.x = (float)L;
                v.y = (float)(L - (double)v.x);
            }
            len[slot] = v;
        }
    }
}

__global__ void k_dw_split(const double* __restrict__ in, int64_t count, float2* __restrict__ out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        const float h = (float)in[k];
        out[k] = make_float2(h, (float)(in[k] - (double)h));
    }
}

int grid_of(int64_t work)
{
    const int64_t b = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace

#if PD_DW_VV
#define PD_DW_KERNELS step_dw_kernels_vv
#else
#define PD_DW_KERNELS step_dw_kernels_ec
#endif
// the kernel variants of this build: [sc_mode][uniform weights][softening]
const void* PD_DW_KERNELS(int sc_mode, bool uniform_w, bool soft)
{
    static const void* const k[8] = {
        (const void*)k_step_dw<0, false, false>, (const void*)k_step_dw<0, false, true>,
        (const void*)k_step_dw<0, true, false>,  (const void*)k_step_dw<0, true, true>,
        (const void*)k_step_dw<1, false, false>, (const void*)k_step_dw<1, false, true>,
        (const void*)k_step_dw<1, true, false>,  (const void*)k_step_dw<1, true, true>};
    return k[(sc_mode ? 4 : 0) + (uniform_w ? 2 : 0) + (soft ? 1 : 0)];
}
#undef PD_DW_KERNELS

#if !PD_DW_VV
const void* step_dw_kernels_vv(int sc_mode, bool uniform_w, bool soft);

const void* step_dw_kernel(int sc_mode, bool uniform_w, bool soft, bool vv)
{
    return vv ? step_dw_kernels_vv(sc_mode, uniform_w, soft)
              : step_dw_kernels_ec(sc_mode, uniform_w, soft);
}

cudaError_t launch_step_dw(const StepArgsF64& a, const DwArgs& d, int sc_mode, int grid, int block,
                           cudaStream_t s)
{
    const void* fn = step_dw_kernel(sc_mode, d.uniform_w != 0, a.integ != nullptr,
                                    a.vv != 0 || a.peek != 0);
    void* args[] = {const_cast<StepArgsF64*>(&a), const_cast<DwArgs*>(&d)};
    return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, 0, s);
}

cudaError_t launch_dw_publish(const double* rec64, float4* rec, int64_t n_pad, const double* origin,
                              double inv_delta, cudaStream_t s)
{
    k_dw_publish<<<grid_of(n_pad), 256, 0, s>>>(rec64, rec, n_pad, origin[0], origin[1], origin[2],
                                                inv_delta);
    return cudaGetLastError();
}

cudaError_t launch_dw_len(const double* x64, const int32_t* nbr, int64_t n, int Q,
                          double inv_delta, float2* len, cudaStream_t s)
{
    k_dw_len<<<grid_of(((n + 31) >> 5) << 5), 256, 0, s>>>(x64, nbr, n, Q, inv_delta, len);
    return cudaGetLastError();
}

cudaError_t launch_dw_split(const double* in, int64_t count, float2* out, cudaStream_t s)
{
    k_dw_split<<<grid_of(count), 256, 0, s>>>(in, count, out);
    return cudaGetLastError();
}

#endif  // !PD_DW_VV

}  // namespace pd
