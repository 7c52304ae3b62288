// Ordinary state-based model (the linear peridynamic solid, section
// "State-based Peridynamics"; the FP64 form and the formulas are in
// pd_step_osb.cu) on a regular lattice: the two loops of the step as stencil
// kernels over the lattice layout of pd_step_f32_lat.cu (no neighbour ids,
// xi = kappa o, FP64 displacement published to the bond arithmetic rounded to
// FP32).  Lengths in horizon units; with m~_i = sum_j |xi~|^2 V_j the weighted
// volume in horizon units (fixed, the family after the cuts):
//   theta_i = (3 / m~_i) sum_j mu_ij |xi~| e~ V_j           (dilation loop)
//   A_i = (3K - 5G) theta_i / (delta m~_i),  B_i = 15 G / (delta m~_i)
//   F_i = sum_j mu_ij ((A_i + A_j) |xi~| + (B_i + B_j) e~) V_j y / |y|   (force loop)
// which is t_ij + t_ji of the linear solid (alpha = 3K theta / m - beta theta / 3,
// beta = 15 G / m) with m = delta^2 m~.  The extension comes without
// cancellation: e~ = |y| - |xi| = num / (|xi| + |y|), num = |y|^2 - |xi|^2.
// Bonds break in the dilation loop (Eq. 6 with s = e / |xi|), with the bond
// step's near-s_c decision, so a bond that breaks in a step enters neither
// loop; the dilation kernel also writes the damage (Eq. 8) and, for the
// force loop, a 16-byte record per node {h, A}; B, fixed, is read from a
// per-node array beside it (16 + 4 bytes per neighbour).
#define PD_LAT_HELPERS 1
#include "pd_step_f32_lat.cu"

namespace pd {
namespace {

// A node's state over a stencil walk of either loop.
struct OsbNode {
    LatOwn own;
    int64_t i;
    float acc;          // dilation: sum |xi~| e~ over intact bonds (x V at the end)
    float2 fxy;         // force: sum of the bonds' terms (x V at the end), (x, y) paired
    float fz;
    float A, B;         // force: the node's own coefficients
    uint32_t word[4];   // bond flags
    uint32_t pend;      // dilation: near-s_c candidates of the current flag word
    int alive;
};

// The dilation term |xi| e~ of a candidate bond to offset (ox, oy, oz), from the
// published displacements: the walk's series term (as the walk forms it) and,
// in *exact, the exact |xi| num / (|xi| + |y|)
__device__ __forceinline__ float osb_dil_term_rt(const StepArgsF32& a, const float4* P, int64_t i,
                                                 int64_t j, int ox, int oy, int oz, int q,
                                                 float* exact)
{
    LatOwn own;
    const float4 hi = ld_pub(P + i);
    own.nxy = make_float2(-hi.x, -hi.y);
    own.nz = -hi.z;
    const float3 e = lat_eta(own, ld_pub(P + j));
    const float num = fmaf(e.x, e.x + a.lat_xi2[ox + 3],
                           fmaf(e.y, e.y + a.lat_xi2[oy + 3], e.z * (e.z + a.lat_xi2[oz + 3])));
    const float y2 = num + a.lat_q[q];
    const float ay = y2 * rsqrt_fast(y2);
    *exact = fabsf(num) > a.lat_pt[q] ? a.lat_l[q] * (num * rcp_fast(a.lat_l[q] + ay)) : 0.0f;
    return num * fmaf(fmaf(a.lat_dc[2][q], num, a.lat_dc[1][q]), num, a.lat_dc[0][q]);
}

template <int SCM>
__device__ __noinline__ float osb_resolve(const StepArgsF32& a, int cur, int64_t i, int m,
                                          bool* broken)
{
    const int ox = c_stencil.o[m][0], oy = c_stencil.o[m][1], oz = c_stencil.o[m][2];
    const int q = c_stencil.o[m][3];
    const int64_t j = i + (int64_t)ox * a.lat_sx + (int64_t)oy * a.lat_sy + oz;
    const double sc = SCM == 1 ? sc_draw(a.sc_seed, a.sc_lo, a.sc_hi, a.gid[i], a.gid[j]) : a.sc;
    const bool brk = lat_breaks(a, cur, i, j, ox, oy, oz, q, sc);
    *broken = brk;
    // the correction of the term the walk added: all of it back when the bond
    // breaks, exact minus series past the series' range (|num| > pt)
    float exact;
    const float ser = osb_dil_term_rt(a, a.lat_pub[cur], i, j, ox, oy, oz, q, &exact);
    if (brk) return -ser;
    return exact != 0.0f ? exact - ser : 0.0f;  // exact is formed past the range only
}

// Bond K of a row with q_xy = QXY (see lat_row_bond): KIND 0 the dilation loop
// (Prow: published records), 1 the force loop (Prow: 16-byte state-based records
// {h, A}, Brow: B); xi, xi2: the (x, y) components of xi and 2 xi of the row,
// which go through paired FP32 instructions.
template <int KIND, int QXY, int K, int ZX, int ZY>
__device__ __forceinline__ void osb_row_bond(const StepArgsF32& a, float2 xi, float2 xi2,
                                             const float4* Prow, const float* Brow,
                                             uint32_t rb, uint32_t& rp, OsbNode& s)
{
    constexpr int OZ = stencil_row_oz(QXY, K);
    constexpr int Q = QXY + OZ * OZ;
    const float4 h = ld_pub(Prow + OZ);  // dilation: {h, 0}; force: {h, A_j}
    const float2 exy = __fadd2_rn(make_float2(h.x, h.y), s.own.nxy);
    const float ez = h.z + s.own.nz;
    const float2 txy = (ZX && ZY) ? exy : __fadd2_rn(exy, xi2);
    const float tz = OZ ? ez + a.lat_xi2[OZ + 3] : ez;
    const bool alive = (rb >> K) & 1u;
    // dilation loop: an absent or broken bond enters with num = 0 (no term and no
    // candidate); near-s_c candidates keep their term, the ones that break give
    // it back after the flag word
    const float num0 = fmaf(exy.x, txy.x, fmaf(exy.y, txy.y, ez * tz));
    const float num = (KIND == 0 && !alive) ? 0.0f : num0;
    if constexpr (KIND == 0) {
        // |xi| e~ from its series in x = num / |xi|^2 (no square root or division);
        // the candidates (the near-s_c band and |x| past the series) are decided and
        // corrected after the flag word
        s.acc += num * fmaf(fmaf(a.lat_dc[2][Q], num, a.lat_dc[1][Q]), num, a.lat_dc[0][Q]);
        const bool cand = fabsf(num - a.lat_cc[Q]) >= a.lat_ch[Q];
        rp |= cand ? (1u << K) : 0u;
    } else {
        const float y2 = num + a.lat_q[Q];
        const float ry = rsqrt_fast(y2);
        const float ay = y2 * ry;
        const float ext = num * rcp_fast(a.lat_l[Q] + ay);  // e~ = |y| - |xi|
        const float t = (s.A + h.w) * a.lat_l[Q] + (s.B + ld_f32(Brow + OZ)) * ext;
        const float f = alive ? t * ry : 0.0f;
        const float2 yxy = (ZX && ZY) ? exy : __fadd2_rn(exy, xi);
        const float yz = OZ ? ez + a.lat_xi[OZ + 3] : ez;
        s.fxy = __ffma2_rn(make_float2(f, f), yxy, s.fxy);
        s.fz = fmaf(f, yz, s.fz);
    }
}

template <int KIND, int SG, int R, int... K>
__device__ __forceinline__ void osb_row_fixed(const StepArgsF32& a, const float4* Pi,
                                              const float* Bi, OsbNode& s,
                                              std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr Off3 o = stencil_row_xy(sg.qxy, sg.row0 + R);
    constexpr int b0 = sg.bit0 + stencil_row_len(sg.qxy) * R;
    const int off = o.x * a.lat_sx + o.y * a.lat_sy;
    const uint32_t rb = s.word[sg.word] >> b0;
    uint32_t rp = 0u;
    const float2 xi = make_float2(a.lat_xi[o.x + 3], a.lat_xi[o.y + 3]);
    const float2 xi2 = make_float2(a.lat_xi2[o.x + 3], a.lat_xi2[o.y + 3]);
    (osb_row_bond<KIND, sg.qxy, K, o.x == 0, o.y == 0>(a, xi, xi2, Pi + off,
                                                       KIND == 1 ? Bi + off : nullptr, rb, rp, s),
     ...);
    if (KIND == 0) s.pend |= rp << b0;
}

template <int KIND, int SG, int... R>
__device__ __forceinline__ void osb_rows_fixed(const StepArgsF32& a, const float4* Pi,
                                               const float* Bi, OsbNode& s,
                                               std::integer_sequence<int, R...>)
{
    (osb_row_fixed<KIND, SG, R>(
         a, Pi, Bi, s, std::make_integer_sequence<int, stencil_row_len(stencil_seg(SG).qxy)>{}),
     ...);
}

template <int KIND, int SG, int... K>
__device__ __forceinline__ void osb_rows_loop(const StepArgsF32& a, const float4* Pi,
                                              const float* Bi, OsbNode& s,
                                              std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
#pragma unroll 1
    for (int r = 0; r < sg.nrows; ++r) {
        const float4 xr = a.lat_rxi[sg.first + r];
        const int off = a.lat_roff[sg.first + r];
        const int b0 = sg.bit0 + len * r;
        const uint32_t rb = s.word[sg.word] >> b0;
        uint32_t rp = 0u;
        (osb_row_bond<KIND, sg.qxy, K, sg.zx, sg.zy>(a, make_float2(xr.x, xr.y),
                                                     make_float2(xr.z, xr.w), Pi + off,
                                                     KIND == 1 ? Bi + off : nullptr, rb, rp, s),
         ...);
        if (KIND == 0) s.pend |= rp << b0;
    }
}

template <int KIND, int SG>
__device__ __forceinline__ void osb_seg(const StepArgsF32& a, const float4* Pi, const float* Bi,
                                        OsbNode& s)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    if constexpr (sg.unroll)
        osb_rows_fixed<KIND, SG>(a, Pi, Bi, s, std::make_integer_sequence<int, sg.nrows>{});
    else
        osb_rows_loop<KIND, SG>(a, Pi, Bi, s,
                                std::make_integer_sequence<int, stencil_row_len(sg.qxy)>{});
}

// dilation loop: after flag word W, decide its near-s_c candidates
template <int SCM, int W>
__device__ __forceinline__ void osb_word_end(const StepArgsF32& a, int cur, OsbNode& s)
{
    uint32_t nword = s.word[W];
    uint32_t pend = s.pend;
    while (pend) {
        const int bb = __ffs(pend) - 1;
        pend &= pend - 1u;
        bool broken;
        const float c = osb_resolve<SCM>(a, cur, s.i, 32 * W + bb, &broken);
        if (broken) nword &= ~(1u << bb);
        s.acc += c;  // the candidate's correction (osb_resolve)
    }
    s.word[W] = nword;
    s.alive += __popc(nword);
    s.pend = 0u;
}

template <int KIND, int SCM>
__device__ __forceinline__ void osb_walk(const StepArgsF32& a, int cur, const float4* Pi,
                                         const float* Bi, OsbNode& s)
{
    osb_seg<KIND, 0>(a, Pi, Bi, s);
    osb_seg<KIND, 1>(a, Pi, Bi, s);
    osb_seg<KIND, 2>(a, Pi, Bi, s);
    if constexpr (KIND == 0) osb_word_end<SCM, 0>(a, cur, s);
    osb_seg<KIND, 3>(a, Pi, Bi, s);
    osb_seg<KIND, 4>(a, Pi, Bi, s);
    osb_seg<KIND, 5>(a, Pi, Bi, s);
    if constexpr (KIND == 0) osb_word_end<SCM, 1>(a, cur, s);
    osb_seg<KIND, 6>(a, Pi, Bi, s);
    osb_seg<KIND, 7>(a, Pi, Bi, s);
    osb_seg<KIND, 8>(a, Pi, Bi, s);
    if constexpr (KIND == 0) osb_word_end<SCM, 2>(a, cur, s);
    osb_seg<KIND, 9>(a, Pi, Bi, s);
    if constexpr (KIND == 0) osb_word_end<SCM, 3>(a, cur, s);
}

// the dilation loop: breaks, theta, damage and the force loop's records
template <int SCM>
__global__ void __launch_bounds__(PD_LAT_THREADS, PD_LAT_MIN_BLOCKS)
    k_osb_lat_dilation(const __grid_constant__ StepArgsF32 a, const OsbLatArgs o)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const int cur = (int)(step & 1);
    const int64_t nslices = (a.n + 31) >> 5;
    const float4* __restrict__ P = a.lat_pub[cur];
    for (int64_t g = wid; g < nslices; g += nwarps) {
        OsbNode s;
        s.i = (g << 5) + lane;
        const float4 hi = ld_pub(P + s.i);
        s.own.nxy = make_float2(-hi.x, -hi.y);
        s.own.nz = -hi.z;
        uint32_t* bw = a.bits + g * 4 * 32 + lane;
        uint32_t w0[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w0[q] = s.word[q] = bw[q * 32];
        s.acc = 0.f;
        s.pend = 0u;
        s.alive = 0;
        osb_walk<0, SCM>(a, cur, P + s.i, nullptr, s);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (s.word[q] != w0[q]) bw[q * 32] = s.word[q];
        const int64_t i = s.i;
        if (i >= a.n) continue;
        const float4 c = o.coef[i];  // {3 / m~, (3K - 5G) / (delta m~), 15 G / (delta m~)}
        const float theta = c.x * a.w_const * s.acc;
        o.theta[i] = theta;
        o.rec[i] = make_float4(hi.x, hi.y, hi.z, c.y * theta);
        const float wi = a.wsum_inv[i];
        const float ws = a.w_const * (float)s.alive;
        a.damage[i] = wi > 0.0f ? fmaxf(0.0f, 1.0f - ws * wi) : 0.0f;
    }
}

// the force loop and the node's update (FP32 force, FP64 u, as the bond step)
__global__ void __launch_bounds__(PD_LAT_THREADS, PD_LAT_MIN_BLOCKS)
    k_osb_lat_force(const __grid_constant__ StepArgsF32 a, const OsbLatArgs o)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const int cur = (int)(step & 1);
    const int64_t nslices = (a.n + 31) >> 5;
    float4* __restrict__ Pout = const_cast<float4*>(a.lat_pub[cur ^ 1]);
    const double* __restrict__ U = a.lat_u[cur];
    double* __restrict__ Uout = a.lat_u[cur ^ 1];
    const float4* __restrict__ S = o.rec;
    for (int64_t g = wid; g < nslices; g += nwarps) {
        OsbNode s;
        s.i = (g << 5) + lane;
        const float4 r0 = ld_pub(S + s.i);
        s.own.nxy = make_float2(-r0.x, -r0.y);
        s.own.nz = -r0.z;
        s.A = r0.w;
        s.B = o.bco[s.i];
        const uint32_t* bw = a.bits + g * 4 * 32 + lane;
#pragma unroll
        for (int q = 0; q < 4; ++q) s.word[q] = bw[q * 32];
        s.fxy = make_float2(0.f, 0.f);
        s.fz = 0.f;
        osb_walk<1, 0>(a, cur, S + s.i, o.bco + s.i, s);
        const int64_t i = s.i;
        if (i >= a.n) continue;
        const float V = a.w_const;  // the volume (uniform)
        const uint32_t cls = a.bcc[i];
        uint32_t mask = 0u;
        const BcClass* bc = nullptr;
        float F[3] = {V * s.fxy.x, V * s.fxy.y, V * s.fz};
        if (cls != 0u) {
            bc = a.bct + cls;
            mask = bc->mask;
#pragma unroll
            for (int c = 0; c < 3; ++c) F[c] += (float)(a.load * bc->force[c]);
        }
        double un[3];
        bool finite = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float vi = a.v[3 * i + c];
            float vn = vi + a.dt_f * (F[c] - a.eta_f * vi) / a.rho_f;
            un[c] = fma((double)vn, (double)a.dtd_f, U[3 * i + c]);
            if (mask & (1u << c)) {
                const double s_now = a.disp_rate * (double)step;
                const double s_next = a.disp_rate * (double)(step + 1);
                un[c] = bc->disp[c] * s_next * a.inv_delta;
                vn = (float)(bc->disp[c] * (s_next - s_now) / a.dt);
            }
            finite = finite && isfinite(un[c]);
            a.v[3 * i + c] = vn;
            Uout[3 * i + c] = un[c];
        }
        Pout[i] = make_float4((float)un[0], (float)un[1], (float)un[2], 0.0f);
        if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
    }
}

}  // namespace

const void* osb_lat_force_kernel() { return (const void*)k_osb_lat_force; }
const void* osb_lat_dilation_kernel(int sc_mode)
{
    return sc_mode == 0 ? (const void*)k_osb_lat_dilation<0> : (const void*)k_osb_lat_dilation<1>;
}

cudaError_t launch_osb_lat_step(const StepArgsF32& a, const OsbLatArgs& o, int sc_mode, int grid,
                                int block, cudaStream_t s)
{
    if (sc_mode == 0)
        k_osb_lat_dilation<0><<<grid, block, 0, s>>>(a, o);
    else
        k_osb_lat_dilation<1><<<grid, block, 0, s>>>(a, o);
    if (cudaPeekAtLastError() == cudaSuccess) k_osb_lat_force<<<grid, block, 0, s>>>(a, o);
    return cudaGetLastError();
}

}  // namespace pd
