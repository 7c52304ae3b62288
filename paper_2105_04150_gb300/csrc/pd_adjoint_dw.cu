// Reverse step of the adjoint in double-word FP32 arithmetic, for handles
// created with PD_PREC_DW; it computes what the FP64 reverse step (k_adj_step
// in pd_adjoint.cu) computes:
//
//   ubar^n_m = ubar_m + (dt/rho) sum_j c_mj K_mj d_mj,  d_mj = V_m w_j - V_j w_m
//   vbar^n_m = (1 - dt eta/rho) w_m
//   dL/dc[m->j] += (dt/rho) s V_j (y/|y|).w_m
//
// with K = (1/L - 1/|y|) I + y y^T / |y|^3, the derivative of s y/|y| (Eqs.
// 4-5) in y = xi + eta.  Lengths are in units of the horizon delta, so that
// K = (1/delta) [(1/L~ - 1/r~) I + y~ y~^T / r~^3]; the 1/delta, the dt/rho
// and (uniform volumes) V are applied once per node, c_mj per bond.
// Per step, k_adj_mask_publish_dw forms w and writes double-word copies of u^n
// and w for the neighbours; k_adj_step_dw walks the sliced family
// like the forward kernels (two slots per iteration, masked slots dropped by
// selects) and keeps the per-slot stiffness gradient as a double-word
// accumulator that k_adj_merge_dw scales by dt/rho into the FP64 result.
#include <cuda_runtime.h>

#include "pd_dw.h"
#include "pd_internal.h"

namespace pd {
namespace {

using namespace dwa;

int grid_of(int64_t work)
{
    const int64_t b = (work + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

__device__ __forceinline__ void split(double x, float& h, float& l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

// Start of a reverse step for node p: w = ws (vbar + dt ubar) with the
// controlled components of ubar and vbar zeroed (as k_adj_mask), and the double-word
// records the bond loop reads: positions copied from the forward double-word
// records, u^n / delta and V as the forward kernel has them ({xh, uh.x}
// {uh.y, uh.z, Vh, Vl} {xl, ul.x} {ul.y, ul.z, 0, 0}), and w ({wh, wl.x}
// {wl.y, wl.z, 0, 0}).
__global__ void k_adj_mask_publish_dw(const double* __restrict__ ub, const double* __restrict__ vb,
                                      const uint8_t* __restrict__ bcc,
                                      const BcClass* __restrict__ bct, double dt, double ws,
                                      const float4* __restrict__ fwd,
                                      const double* __restrict__ un,
                                      const double* __restrict__ vol, int64_t n_pad,
                                      double inv_delta, double* __restrict__ ubm,
                                      double* __restrict__ w, float4* __restrict__ rec,
                                      float4* __restrict__ wrec)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n_pad;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t cls = bcc[p];
        const uint32_t mask = cls ? bct[cls].mask : 0u;
        const float4 a0 = fwd[4 * p], b0 = fwd[4 * p + 2];
        float uh[3], ul[3], wh[3], wl[3], vh, vl;
        for (int k = 0; k < 3; ++k) {
            const bool ctl = (mask >> k) & 1u;
            const double u = ctl ? 0.0 : ub[3 * p + k];
            const double v = ctl ? 0.0 : vb[3 * p + k];
            const double wk = ws * (v + dt * u);
            ubm[3 * p + k] = u;
            w[3 * p + k] = wk;
            split(un[3 * p + k] * inv_delta, uh[k], ul[k]);
            split(wk, wh[k], wl[k]);
        }
        split(vol[p], vh, vl);
        rec[4 * p] = make_float4(a0.x, a0.y, a0.z, uh[0]);
        rec[4 * p + 1] = make_float4(uh[1], uh[2], vh, vl);
        rec[4 * p + 2] = make_float4(b0.x, b0.y, b0.z, ul[0]);
        rec[4 * p + 3] = make_float4(ul[1], ul[2], 0.0f, 0.0f);
        wrec[2 * p] = make_float4(wh[0], wh[1], wh[2], wl[0]);
        wrec[2 * p + 1] = make_float4(wl[1], wl[2], 0.0f, 0.0f);
    }
}

struct AdjBond {
    Dw f[3];  // c (k1 d + k2 y), the node's common factors left out
    Dw g;     // s V_j (y/|y|).w_m, the bond's dL/dc without dt/rho
};

// One bond m -> j of the reverse step.  UW: uniform volumes, d = V (w_j - w_m)
// with V applied by the caller; otherwise d = V_m w_j - V_j w_m.
template <bool UW>
__device__ __forceinline__ AdjBond adj_bond(const OwnDw& o, const Dw (&wm)[3], Dw Vm,
                                            const Rec& j, const float4 wj0, const float4 wj1,
                                            const float2 len, Dw cij)
{
    const float jxh[3] = {j.a0.x, j.a0.y, j.a0.z}, juh[3] = {j.a0.w, j.a1.x, j.a1.y};
    const float jxl[3] = {j.b0.x, j.b0.y, j.b0.z}, jul[3] = {j.b0.w, j.b1.x, j.b1.y};
    const Dw wj[3] = {{wj0.x, wj0.w}, {wj0.y, wj1.x}, {wj0.z, wj1.y}};
    const Dw Vj{j.a1.z, j.a1.w};
    Dw y[3], d[3], nm[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const Dw xi{jxh[c] - o.xh[c], jxl[c] - o.xl[c]};  // exact leading difference
        Dw et = two_sum(juh[c], -o.uh[c]);
        et.l += jul[c] - o.ul[c];
        y[c] = dw_add(xi, et);
        nm[c] = dw_mul(et, dw_add(xi, y[c]));  // eta_c (2 xi_c + eta_c)
        if (UW) {
            d[c] = two_sum(wj[c].h, -wm[c].h);
            d[c].l += wj[c].l - wm[c].l;
        } else {
            const Dw a = dw_mul(Vm, wj[c]), b = dw_mul(Vj, wm[c]);
            d[c] = dw_add(a, Dw{-b.h, -b.l});
        }
    }
    // the stretch as in the forward kernel, s = num / (L (L + |y|)) with
    // num = |y|^2 - L^2 free of cancellation (the difference |y| / L - 1 would
    // carry the positions' rounding as an absolute error), and
    // 1/L - 1/|y| = s / |y|
    Dw num = two_sum(nm[0].h, nm[1].h);
    num.l += nm[0].l + nm[1].l;
    num = dw_add(num, nm[2]);
    const Dw L{len.x, len.y};
    Dw r, ir;
    dw_norm(dw_add(dw_mul(L, L), num), r, ir);
    const Dw s = dw_div(num, dw_mul(L, dw_add(L, r)));
    Dw yd = dw_mul(y[0], d[0]);
    yd = dw_add(yd, dw_mul(y[1], d[1]));
    yd = dw_add(yd, dw_mul(y[2], d[2]));
    const Dw k1 = dw_mul(cij, dw_mul(s, ir));
    const Dw k2 = dw_mul(cij, dw_mul(yd, dw_mul(ir, dw_mul(ir, ir))));
    AdjBond out;
#pragma unroll
    for (int c = 0; c < 3; ++c) out.f[c] = dw_add(dw_mul(k1, d[c]), dw_mul(k2, y[c]));
    Dw yw = dw_mul(y[0], wm[0]);
    yw = dw_add(yw, dw_mul(y[1], wm[1]));
    yw = dw_add(yw, dw_mul(y[2], wm[2]));
    out.g = dw_mul(dw_mul(s, Vj), dw_mul(yw, ir));
    return out;
}

template <bool UW>
__global__ void __launch_bounds__(256, 2) k_adj_step_dw(const __grid_constant__ AdjDwArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int Q = a.Q;
    const int64_t W = 32LL * Q;
    const int64_t nslices = (a.n + 31) >> 5;
    const Dw c_const{a.c.x, a.c.y};
    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int64_t m = (g << 5) + lane;
        const int Wg = a.sw[g];
        const int32_t* __restrict__ col = a.nbr + g * W * 32 + lane;
        Rec me;
        ld_rec(a.rec + 4 * m, me.a0, me.a1);
        ld_rec(a.rec + 4 * m + 2, me.b0, me.b1);
        const OwnDw own = own_of(me);
        float4 w0, w1;
        ld_rec(a.wrec + 2 * m, w0, w1);
        const Dw wm[3] = {{w0.x, w0.w}, {w0.y, w1.x}, {w0.z, w1.y}};
        const Dw Vm{me.a1.z, me.a1.w};
        Dw acc[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        // chunks of two slots, ids one chunk ahead, each flag word read once
        const int nch = (Wg + 1) >> 1;
        int32_t jn0 = __ldg(col), jn1 = __ldg(col + 32);
        uint32_t word = 0u;
        for (int c = 0; c < nch; ++c) {
            const int m0 = 2 * c;
            const int q = m0 >> 5, b0 = m0 & 31;
            if (b0 == 0) word = a.bits[(g * Q + q) * 32 + lane];
            const int32_t jj[2] = {jn0, jn1};
            if (c + 1 < nch) {
                jn0 = __ldg(col + (m0 + 2) * 32);
                jn1 = __ldg(col + (m0 + 3) * 32);
            }
            const uint32_t wb = word >> b0;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int64_t slot = (g * W + m0 + u) * 32 + lane;
                const int64_t j = jj[u];
                Rec nb;
                ld_rec(a.rec + 4 * j, nb.a0, nb.a1);
                ld_rec(a.rec + 4 * j + 2, nb.b0, nb.b1);
                float4 v0, v1;
                ld_rec(a.wrec + 2 * j, v0, v1);
                const float2 len = __ldg(a.len + slot);
                Dw cij = c_const;
                if (a.cb != nullptr) {  // per-bond stiffness (a uniform branch)
                    const float2 cv = __ldg(a.cb + slot);
                    cij = Dw{cv.x, cv.y};
                }
                const AdjBond bd = adj_bond<UW>(own, wm, Vm, nb, v0, v1, len, cij);
                // masked slots (broken, or no bond: neighbour = the node itself,
                // non-finite terms) are dropped by selects
                const bool ok = (wb >> u) & 1u;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const Dw t = two_sum(acc[k].h, ok ? bd.f[k].h : 0.0f);
                    acc[k].h = t.h;
                    acc[k].l += t.l + (ok ? bd.f[k].l : 0.0f);
                }
                if (ok) {
                    const float2 old = a.gc[slot];
                    const Dw t = two_sum(old.x, bd.g.h);
                    a.gc[slot] = make_float2(t.h, old.y + (t.l + bd.g.l));
                }
            }
        }
        if (m < a.n) {
            const double wd[3] = {a.w[3 * m], a.w[3 * m + 1], a.w[3 * m + 2]};
            const double scale = a.dt_rho * a.inv_delta * (UW ? a.vol0 : 1.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                a.ub_out[3 * m + k] =
                    a.ubm[3 * m + k] + scale * ((double)acc[k].h + (double)acc[k].l);
                a.vb_out[3 * m + k] = a.damp * wd[k];
            }
            const uint32_t cls = a.bcc[m];
            if (cls) {
                const BcClass& bc = a.bct[cls];
                a.gl[m] += bc.force[0] * wd[0] + bc.force[1] * wd[1] + bc.force[2] * wd[2];
            }
        }
    }
}

// gc (FP64) = dt/rho times the double-word per-slot accumulator
__global__ void k_adj_merge_dw(const float2* __restrict__ acc, int64_t count, double scale,
                               double* __restrict__ gc)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x)
        gc[k] = scale * ((double)acc[k].x + (double)acc[k].y);
}

}  // namespace

cudaError_t launch_adj_mask_publish_dw(const double* ub, const double* vb, const uint8_t* bcc,
                                       const BcClass* bct, double dt, double ws,
                                       const float4* fwd, const double* un, const double* vol,
                                       int64_t n_pad, double inv_delta, double* ubm, double* w,
                                       float4* rec, float4* wrec, cudaStream_t s)
{
    k_adj_mask_publish_dw<<<grid_of(n_pad), 256, 0, s>>>(ub, vb, bcc, bct, dt, ws, fwd, un, vol, n_pad,
                                                         inv_delta, ubm, w, rec, wrec);
    return cudaGetLastError();
}

cudaError_t launch_adj_step_dw(const AdjDwArgs& a, int grid, int block, cudaStream_t s)
{
    if (a.uniform_w)
        k_adj_step_dw<true><<<grid, block, 0, s>>>(a);
    else
        k_adj_step_dw<false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_adj_merge_dw(const float2* acc, int64_t count, double scale, double* gc,
                                cudaStream_t s)
{
    k_adj_merge_dw<<<grid_of(count), 256, 0, s>>>(acc, count, scale, gc);
    return cudaGetLastError();
}

}  // namespace pd
