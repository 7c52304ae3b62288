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
// per-node array beside it (16 + 4 bytes per neighbour).  Both loops walk the
// stencil two bonds at a time (paired FP32 instructions, as the bond-based
// walk) and take their per-bond functions of x = num / |xi|^2 from series to
// x^2 (within 0.25 ulp for |x| <= kLatPolyX): the dilation term |xi| e~, whose
// candidates past that range are corrected exactly after each flag word, and
// the force loop's |xi| / |y| and e~ / |y|, which a slice of 32 nodes takes
// from the series unless the dilation loop found a candidate among its bonds
// (then every bond of the slice is formed exactly, one at a time).
#define PD_LAT_HELPERS 1
#include "pd_step_f32_lat.cu"

namespace pd {
namespace {

// A node's state over the dilation loop's walk.  It takes its bonds two at a
// time (osb_pair_bond): the first half of each register pair belongs to the
// first bond of a pair, the second half to the second.
struct OsbNode {
    float2 nx, ny, nz;  // the lane's own published displacement, negated, twice
    int64_t i;
    float2 acc;         // sums of |xi~| e~ over intact bonds (x V at the end)
    uint32_t word[4];   // bond flags
    uint32_t pend;      // near-s_c candidates of the current flag word
    uint32_t anyc;      // nonzero: the walk had a candidate
    int alive;
};

// A node's state over the force loop's walk: in pairs of bonds with the
// series factors (osb_force_pair), or one bond at a time with the exact ones
// (osb_force_bond, its (x, y) components paired)
struct OsbForceNode {
    float2 nx, ny, nz;  // the lane's own published displacement, negated, twice
    LatOwn own;         // the same, for the one-bond walk
    int64_t i;
    float2 fx, fy, fz;  // pair walk: force sums over the first and second bonds of the pairs
    float2 fxy;         // one-bond walk: force sum, (x, y) paired
    float fzs;
    float A, B;         // the node's own coefficients
    uint32_t word[4];   // bond flags
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

// Dilation loop: two bonds of equal |xi| walked together, as in the bond-based
// walk (lat_pair_bond): bond K0 of the row at P0 (flags rb0, candidates rp0)
// and bond K1 of the row at P1 (rb1, rp1), P the published records; xi2x,
// xi2y: the rows' x and y components of 2 xi (ZX / ZY: 0 in both).  Each half
// of a paired instruction is rounded as the scalar operation, so each bond's
// term is that of the one-bond formula (osb_dil_term_rt re-forms it).
template <int QXY, int K0, int K1, int ZX, int ZY>
__device__ __forceinline__ void osb_dil_pair(const StepArgsF32& a, const float2 xi2x,
                                             const float2 xi2y, const float4* P0,
                                             const float4* P1, uint32_t rb0, uint32_t rb1,
                                             uint32_t& rp0, uint32_t& rp1, OsbNode& s)
{
    constexpr int OZ0 = stencil_row_oz(QXY, K0), OZ1 = stencil_row_oz(QXY, K1);
    static_assert(OZ0 * OZ0 == OZ1 * OZ1, "the two bonds of a pair have the same |xi|");
    constexpr int Q = QXY + OZ0 * OZ0;
    const float4 h0 = ld_pub(P0 + OZ0), h1 = ld_pub(P1 + OZ1);
    const float2 ex = __fadd2_rn(make_float2(h0.x, h1.x), s.nx);
    const float2 ey = __fadd2_rn(make_float2(h0.y, h1.y), s.ny);
    const float2 ez = __fadd2_rn(make_float2(h0.z, h1.z), s.nz);
    const float2 tx = ZX ? ex : __fadd2_rn(ex, xi2x);
    const float2 ty = ZY ? ey : __fadd2_rn(ey, xi2y);
    const float2 tz = OZ0 ? __fadd2_rn(ez, make_float2(a.lat_xi2[OZ0 + 3], a.lat_xi2[OZ1 + 3]))
                          : ez;
    // an absent or broken bond enters with num = 0 (no term and no candidate);
    // |xi| e~ from its series in x = num / |xi|^2 (no square root or division);
    // the candidates (the near-s_c band and |x| past the series) keep their term
    // and are decided and corrected after the flag word
    float2 num = __ffma2_rn(ex, tx, __ffma2_rn(ey, ty, __fmul2_rn(ez, tz)));
    num.x = ((rb0 >> K0) & 1u) ? num.x : 0.0f;
    num.y = ((rb1 >> K1) & 1u) ? num.y : 0.0f;
    s.acc = __ffma2_rn(
        num, __ffma2_rn(__ffma2_rn(a.lat_dcd[2][Q], num, a.lat_dcd[1][Q]), num, a.lat_dcd[0][Q]),
        s.acc);
    const float2 d = __fadd2_rn(num, a.lat_ccd[Q]);
    rp0 |= fabsf(d.x) >= a.lat_ch[Q] ? (1u << K0) : 0u;
    rp1 |= fabsf(d.y) >= a.lat_ch[Q] ? (1u << K1) : 0u;
}

// Rows R and R + 1 (compile-time) of segment SG, unrolled, their offsets fixed
template <int SG, int R, int... K>
__device__ __forceinline__ void osb_dil_rowpair_fixed(const StepArgsF32& a, const float4* Pi,
                                                      OsbNode& s, std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    constexpr Off3 o0 = stencil_row_xy(sg.qxy, sg.row0 + R);
    constexpr Off3 o1 = stencil_row_xy(sg.qxy, sg.row0 + R + 1);
    constexpr int b0 = sg.bit0 + len * R;
    const float4* P0 = Pi + (o0.x * a.lat_sx + o0.y * a.lat_sy);
    const float4* P1 = Pi + (o1.x * a.lat_sx + o1.y * a.lat_sy);
    const uint32_t rb0 = s.word[sg.word] >> b0, rb1 = rb0 >> len;
    uint32_t rp0 = 0u, rp1 = 0u;
    const float2 xi2x = make_float2(a.lat_xi2[o0.x + 3], a.lat_xi2[o1.x + 3]);
    const float2 xi2y = make_float2(a.lat_xi2[o0.y + 3], a.lat_xi2[o1.y + 3]);
    (osb_dil_pair<sg.qxy, K, K, o0.x == 0 && o1.x == 0, o0.y == 0 && o1.y == 0>(
         a, xi2x, xi2y, P0, P1, rb0, rb1, rp0, rp1, s),
     ...);
    s.pend |= (rp0 | (rp1 << len)) << b0;
}

template <int SG, int... R>
__device__ __forceinline__ void osb_dil_rows_fixed(const StepArgsF32& a, const float4* Pi,
                                                   OsbNode& s, std::integer_sequence<int, R...>)
{
    (osb_dil_rowpair_fixed<SG, 2 * R>(
         a, Pi, s, std::make_integer_sequence<int, stencil_row_len(stencil_seg(SG).qxy)>{}),
     ...);
}

// The o_x = o_y = 0 row: positions K and len - 1 - K (o_z and -o_z) as pairs
template <int SG, int... K>
__device__ __forceinline__ void osb_dil_row_mirror(const StepArgsF32& a, const float4* Pi,
                                                   OsbNode& s, std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    static_assert(sg.qxy == 0 && sg.nrows == 1 && len % 2 == 0, "the o_x = o_y = 0 row");
    const uint32_t rb = s.word[sg.word] >> sg.bit0;
    uint32_t rp = 0u;
    const float2 z = make_float2(0.f, 0.f);
    (osb_dil_pair<sg.qxy, K, len - 1 - K, 1, 1>(a, z, z, Pi, Pi, rb, rb, rp, rp, s), ...);
    s.pend |= rp << sg.bit0;
}

// Segment SG as a loop over its rows, two rows per iteration
template <int SG, int... K>
__device__ __forceinline__ void osb_dil_rows_loop(const StepArgsF32& a, const float4* Pi,
                                                  OsbNode& s, std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    static_assert(sg.nrows % 2 == 0, "a loop segment walks its rows in pairs");
#pragma unroll 1
    for (int r = 0; r < sg.nrows; r += 2) {
        const int j = sg.first + r;
        const float4 xb = a.lat_rxp[j][1];
        const float4* P0 = Pi + a.lat_roff[j];
        const float4* P1 = Pi + a.lat_roff[j + 1];
        const int b0 = sg.bit0 + len * r;
        const uint32_t rb0 = s.word[sg.word] >> b0, rb1 = rb0 >> len;
        uint32_t rp0 = 0u, rp1 = 0u;
        (osb_dil_pair<sg.qxy, K, K, sg.zx, sg.zy>(a, make_float2(xb.x, xb.y),
                                                  make_float2(xb.z, xb.w), P0, P1, rb0, rb1,
                                                  rp0, rp1, s),
         ...);
        s.pend |= (rp0 | (rp1 << len)) << b0;
    }
}

template <int SG>
__device__ __forceinline__ void osb_dil_seg(const StepArgsF32& a, const float4* Pi, OsbNode& s)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    if constexpr (!sg.unroll)
        osb_dil_rows_loop<SG>(a, Pi, s, std::make_integer_sequence<int, len>{});
    else if constexpr (sg.nrows == 1)
        osb_dil_row_mirror<SG>(a, Pi, s, std::make_integer_sequence<int, len / 2>{});
    else
        osb_dil_rows_fixed<SG>(a, Pi, s, std::make_integer_sequence<int, sg.nrows / 2>{});
}

// after flag word W of the dilation loop, decide its near-s_c candidates
template <int SCM, int W>
__device__ __forceinline__ void osb_word_end(const StepArgsF32& a, int cur, OsbNode& s)
{
    uint32_t nword = s.word[W];
    uint32_t pend = s.pend;
    s.anyc |= pend;
    while (pend) {
        const int bb = __ffs(pend) - 1;
        pend &= pend - 1u;
        bool broken;
        const float c = osb_resolve<SCM>(a, cur, s.i, 32 * W + bb, &broken);
        if (broken) nword &= ~(1u << bb);
        s.acc.x += c;  // the candidate's correction (osb_resolve)
    }
    s.word[W] = nword;
    s.alive += __popc(nword);
    s.pend = 0u;
}

template <int SCM>
__device__ __forceinline__ void osb_dil_walk(const StepArgsF32& a, int cur, const float4* Pi,
                                             OsbNode& s)
{
    osb_dil_seg<0>(a, Pi, s);
    osb_dil_seg<1>(a, Pi, s);
    osb_dil_seg<2>(a, Pi, s);
    osb_word_end<SCM, 0>(a, cur, s);
    osb_dil_seg<3>(a, Pi, s);
    osb_dil_seg<4>(a, Pi, s);
    osb_dil_seg<5>(a, Pi, s);
    osb_word_end<SCM, 1>(a, cur, s);
    osb_dil_seg<6>(a, Pi, s);
    osb_dil_seg<7>(a, Pi, s);
    osb_dil_seg<8>(a, Pi, s);
    osb_word_end<SCM, 2>(a, cur, s);
    osb_dil_seg<9>(a, Pi, s);
    osb_word_end<SCM, 3>(a, cur, s);
}

// Force loop, one bond at a time with the exact factors (the slices of nodes
// with a dilation candidate): bond K of a row with q_xy = QXY (Prow: 16-byte
// state-based records {h, A}, Brow: B); xi, xi2: the (x, y) components of xi
// and 2 xi of the row, which go through paired FP32 instructions.  The bond's
// force factor t / |y| = ((A_i + A_j) |xi| + (B_i + B_j) e~) / |y| with the
// reciprocal square root and the division.
template <int QXY, int K, int ZX, int ZY>
__device__ __forceinline__ void osb_force_bond(const StepArgsF32& a, float2 xi, float2 xi2,
                                               const float4* Prow, const float* Brow, uint32_t rb,
                                               OsbForceNode& s)
{
    constexpr int OZ = stencil_row_oz(QXY, K);
    constexpr int Q = QXY + OZ * OZ;
    const float4 h = ld_pub(Prow + OZ);  // {h, A_j}
    const float2 exy = __fadd2_rn(make_float2(h.x, h.y), s.own.nxy);
    const float ez = h.z + s.own.nz;
    const float2 txy = (ZX && ZY) ? exy : __fadd2_rn(exy, xi2);
    const float tz = OZ ? ez + a.lat_xi2[OZ + 3] : ez;
    const bool alive = (rb >> K) & 1u;
    const float num = fmaf(exy.x, txy.x, fmaf(exy.y, txy.y, ez * tz));
    const float As = s.A + h.w, Bs = s.B + ld_f32(Brow + OZ);
    const float y2 = num + a.lat_q[Q];
    const float ry = rsqrt_fast(y2);
    const float ay = y2 * ry;
    const float ext = num * rcp_fast(a.lat_l[Q] + ay);  // e~ = |y| - |xi|
    const float f0 = (As * a.lat_l[Q] + Bs * ext) * ry;
    const float f = alive ? f0 : 0.0f;
    const float2 yxy = (ZX && ZY) ? exy : __fadd2_rn(exy, xi);
    const float yz = OZ ? ez + a.lat_xi[OZ + 3] : ez;
    s.fxy = __ffma2_rn(make_float2(f, f), yxy, s.fxy);
    s.fzs = fmaf(f, yz, s.fzs);
}

template <int SG, int R, int... K>
__device__ __forceinline__ void osb_force_row_fixed(const StepArgsF32& a, const float4* Pi,
                                                    const float* Bi, OsbForceNode& s,
                                                    std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr Off3 o = stencil_row_xy(sg.qxy, sg.row0 + R);
    constexpr int b0 = sg.bit0 + stencil_row_len(sg.qxy) * R;
    const int off = o.x * a.lat_sx + o.y * a.lat_sy;
    const uint32_t rb = s.word[sg.word] >> b0;
    const float2 xi = make_float2(a.lat_xi[o.x + 3], a.lat_xi[o.y + 3]);
    const float2 xi2 = make_float2(a.lat_xi2[o.x + 3], a.lat_xi2[o.y + 3]);
    (osb_force_bond<sg.qxy, K, o.x == 0, o.y == 0>(a, xi, xi2, Pi + off, Bi + off, rb, s),
     ...);
}

template <int SG, int... R>
__device__ __forceinline__ void osb_force_rows_fixed(const StepArgsF32& a, const float4* Pi,
                                                     const float* Bi, OsbForceNode& s,
                                                     std::integer_sequence<int, R...>)
{
    (osb_force_row_fixed<SG, R>(
         a, Pi, Bi, s, std::make_integer_sequence<int, stencil_row_len(stencil_seg(SG).qxy)>{}),
     ...);
}

template <int SG, int... K>
__device__ __forceinline__ void osb_force_rows_loop(const StepArgsF32& a, const float4* Pi,
                                                    const float* Bi, OsbForceNode& s,
                                                    std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
#pragma unroll 1
    for (int r = 0; r < sg.nrows; ++r) {
        const float4 xr = a.lat_rxi[sg.first + r];
        const int off = a.lat_roff[sg.first + r];
        const uint32_t rb = s.word[sg.word] >> (sg.bit0 + len * r);
        (osb_force_bond<sg.qxy, K, sg.zx, sg.zy>(a, make_float2(xr.x, xr.y),
                                                 make_float2(xr.z, xr.w), Pi + off, Bi + off, rb,
                                                 s),
         ...);
    }
}

template <int SG>
__device__ __forceinline__ void osb_force_seg(const StepArgsF32& a, const float4* Pi,
                                              const float* Bi, OsbForceNode& s)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    if constexpr (sg.unroll)
        osb_force_rows_fixed<SG>(a, Pi, Bi, s, std::make_integer_sequence<int, sg.nrows>{});
    else
        osb_force_rows_loop<SG>(a, Pi, Bi, s,
                                std::make_integer_sequence<int, stencil_row_len(sg.qxy)>{});
}

// Force loop, two bonds of equal |xi| at a time with the series factors (the
// pairs of the dilation loop's walk): bond K0 of the row at P0 (B0: the row's
// B, flags rb0), bond K1 of the row at P1 (B1, rb1)
template <int QXY, int K0, int K1, int ZX, int ZY>
__device__ __forceinline__ void osb_force_pair(const StepArgsF32& a, const float2 xix,
                                               const float2 xiy, const float2 xi2x,
                                               const float2 xi2y, const float4* P0,
                                               const float4* P1, const float* B0, const float* B1,
                                               uint32_t rb0, uint32_t rb1, OsbForceNode& s)
{
    constexpr int OZ0 = stencil_row_oz(QXY, K0), OZ1 = stencil_row_oz(QXY, K1);
    static_assert(OZ0 * OZ0 == OZ1 * OZ1, "the two bonds of a pair have the same |xi|");
    constexpr int Q = QXY + OZ0 * OZ0;
    const float4 h0 = ld_pub(P0 + OZ0), h1 = ld_pub(P1 + OZ1);  // {h, A_j}
    const float2 ex = __fadd2_rn(make_float2(h0.x, h1.x), s.nx);
    const float2 ey = __fadd2_rn(make_float2(h0.y, h1.y), s.ny);
    const float2 ez = __fadd2_rn(make_float2(h0.z, h1.z), s.nz);
    const float2 tx = ZX ? ex : __fadd2_rn(ex, xi2x);
    const float2 ty = ZY ? ey : __fadd2_rn(ey, xi2y);
    const float2 tz = OZ0 ? __fadd2_rn(ez, make_float2(a.lat_xi2[OZ0 + 3], a.lat_xi2[OZ1 + 3]))
                          : ez;
    const float2 num = __ffma2_rn(ex, tx, __ffma2_rn(ey, ty, __fmul2_rn(ez, tz)));
    const float2 As = __fadd2_rn(make_float2(h0.w, h1.w), make_float2(s.A, s.A));
    const float2 Bs = __fadd2_rn(make_float2(ld_f32(B0 + OZ0), ld_f32(B1 + OZ1)),
                                 make_float2(s.B, s.B));
    // |xi| / |y| and e~ / |y| from their series in x = num / |xi|^2
    const float2 p = __ffma2_rn(__ffma2_rn(a.lat_fad[1][Q], num, a.lat_fad[0][Q]), num,
                                make_float2(1.0f, 1.0f));
    const float2 r = __fmul2_rn(
        num, __ffma2_rn(__ffma2_rn(a.lat_fbd[2][Q], num, a.lat_fbd[1][Q]), num, a.lat_fbd[0][Q]));
    float2 f = __ffma2_rn(As, p, __fmul2_rn(Bs, r));
    f.x = ((rb0 >> K0) & 1u) ? f.x : 0.0f;
    f.y = ((rb1 >> K1) & 1u) ? f.y : 0.0f;
    const float2 yx = ZX ? ex : __fadd2_rn(ex, xix);
    const float2 yy = ZY ? ey : __fadd2_rn(ey, xiy);
    const float2 yz = OZ0 ? __fadd2_rn(ez, make_float2(a.lat_xi[OZ0 + 3], a.lat_xi[OZ1 + 3])) : ez;
    s.fx = __ffma2_rn(f, yx, s.fx);
    s.fy = __ffma2_rn(f, yy, s.fy);
    s.fz = __ffma2_rn(f, yz, s.fz);
}

template <int SG, int R, int... K>
__device__ __forceinline__ void osb_force_rowpair_fixed(const StepArgsF32& a, const float4* Pi,
                                                        const float* Bi, OsbForceNode& s,
                                                        std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    constexpr Off3 o0 = stencil_row_xy(sg.qxy, sg.row0 + R);
    constexpr Off3 o1 = stencil_row_xy(sg.qxy, sg.row0 + R + 1);
    constexpr int b0 = sg.bit0 + len * R;
    const int off0 = o0.x * a.lat_sx + o0.y * a.lat_sy;
    const int off1 = o1.x * a.lat_sx + o1.y * a.lat_sy;
    const uint32_t rb0 = s.word[sg.word] >> b0, rb1 = rb0 >> len;
    const float2 xix = make_float2(a.lat_xi[o0.x + 3], a.lat_xi[o1.x + 3]);
    const float2 xiy = make_float2(a.lat_xi[o0.y + 3], a.lat_xi[o1.y + 3]);
    const float2 xi2x = make_float2(a.lat_xi2[o0.x + 3], a.lat_xi2[o1.x + 3]);
    const float2 xi2y = make_float2(a.lat_xi2[o0.y + 3], a.lat_xi2[o1.y + 3]);
    (osb_force_pair<sg.qxy, K, K, o0.x == 0 && o1.x == 0, o0.y == 0 && o1.y == 0>(
         a, xix, xiy, xi2x, xi2y, Pi + off0, Pi + off1, Bi + off0, Bi + off1, rb0, rb1, s),
     ...);
}

template <int SG, int... R>
__device__ __forceinline__ void osb_force_rowpairs_fixed(const StepArgsF32& a, const float4* Pi,
                                                         const float* Bi, OsbForceNode& s,
                                                         std::integer_sequence<int, R...>)
{
    (osb_force_rowpair_fixed<SG, 2 * R>(
         a, Pi, Bi, s, std::make_integer_sequence<int, stencil_row_len(stencil_seg(SG).qxy)>{}),
     ...);
}

template <int SG, int... K>
__device__ __forceinline__ void osb_force_row_mirror(const StepArgsF32& a, const float4* Pi,
                                                     const float* Bi, OsbForceNode& s,
                                                     std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    static_assert(sg.qxy == 0 && sg.nrows == 1 && len % 2 == 0, "the o_x = o_y = 0 row");
    const uint32_t rb = s.word[sg.word] >> sg.bit0;
    const float2 z = make_float2(0.f, 0.f);
    (osb_force_pair<sg.qxy, K, len - 1 - K, 1, 1>(a, z, z, z, z, Pi, Pi, Bi, Bi, rb, rb, s), ...);
}

template <int SG, int... K>
__device__ __forceinline__ void osb_force_rowpairs_loop(const StepArgsF32& a, const float4* Pi,
                                                        const float* Bi, OsbForceNode& s,
                                                        std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    static_assert(sg.nrows % 2 == 0, "a loop segment walks its rows in pairs");
#pragma unroll 1
    for (int r = 0; r < sg.nrows; r += 2) {
        const int j = sg.first + r;
        const float4 xa = a.lat_rxp[j][0], xb = a.lat_rxp[j][1];
        const int off0 = a.lat_roff[j], off1 = a.lat_roff[j + 1];
        const uint32_t rb0 = s.word[sg.word] >> (sg.bit0 + len * r), rb1 = rb0 >> len;
        (osb_force_pair<sg.qxy, K, K, sg.zx, sg.zy>(
             a, make_float2(xa.x, xa.y), make_float2(xa.z, xa.w), make_float2(xb.x, xb.y),
             make_float2(xb.z, xb.w), Pi + off0, Pi + off1, Bi + off0, Bi + off1, rb0, rb1, s),
         ...);
    }
}

template <int SG>
__device__ __forceinline__ void osb_force_pairseg(const StepArgsF32& a, const float4* Pi,
                                                  const float* Bi, OsbForceNode& s)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    if constexpr (!sg.unroll)
        osb_force_rowpairs_loop<SG>(a, Pi, Bi, s, std::make_integer_sequence<int, len>{});
    else if constexpr (sg.nrows == 1)
        osb_force_row_mirror<SG>(a, Pi, Bi, s, std::make_integer_sequence<int, len / 2>{});
    else
        osb_force_rowpairs_fixed<SG>(a, Pi, Bi, s,
                                     std::make_integer_sequence<int, sg.nrows / 2>{});
}

template <int... SG>
__device__ __forceinline__ void osb_force_pairwalk(const StepArgsF32& a, const float4* Pi,
                                                   const float* Bi, OsbForceNode& s,
                                                   std::integer_sequence<int, SG...>)
{
    (osb_force_pairseg<SG>(a, Pi, Bi, s), ...);
}

template <int... SG>
__device__ __forceinline__ void osb_force_walk(const StepArgsF32& a, const float4* Pi,
                                               const float* Bi, OsbForceNode& s,
                                               std::integer_sequence<int, SG...>)
{
    (osb_force_seg<SG>(a, Pi, Bi, s), ...);
}

// the dilation loop: breaks, theta, damage and the force loop's records
template <int SCM>
__global__ void __launch_bounds__(PD_LAT_THREADS, PD_LAT_MIN_BLOCKS)
    k_osb_lat_dilation(const __grid_constant__ StepArgsF32 a, const OsbLatArgs o)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // a direct launch's counter still holds this step (the step's force kernel advances it)
    const int64_t step = a.step_ctr[0] + a.k;
    const int cur = (int)(step & 1);
    const int64_t nslices = (a.n + 31) >> 5;
    const float4* __restrict__ P = a.lat_pub[cur];
    for (int64_t g = wid; g < nslices; g += nwarps) {
        OsbNode s;
        s.i = (g << 5) + lane;
        const float4 hi = ld_pub(P + s.i);
        s.nx = make_float2(-hi.x, -hi.x);
        s.ny = make_float2(-hi.y, -hi.y);
        s.nz = make_float2(-hi.z, -hi.z);
        uint32_t* bw = a.bits + g * 4 * 32 + lane;
        uint32_t w0[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w0[q] = s.word[q] = bw[q * 32];
        s.acc = make_float2(0.f, 0.f);
        s.pend = 0u;
        s.anyc = 0u;
        s.alive = 0;
        osb_dil_walk<SCM>(a, cur, P + s.i, s);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (s.word[q] != w0[q]) bw[q * 32] = s.word[q];
        // the force loop's choice for the slice: exact where a node had a candidate
        const unsigned xs = __ballot_sync(0xffffffffu, s.anyc != 0u);
        if (lane == 0) o.exact[g] = xs != 0u ? 1 : 0;
        const int64_t i = s.i;
        if (i >= a.n) continue;
        const float4 c = o.coef[i];  // {3 / m~, (3K - 5G) / (delta m~), 15 G / (delta m~)}
        const float theta = c.x * a.w_const * (s.acc.x + s.acc.y);
        o.theta[i] = theta;
        o.rec[i] = make_float4(hi.x, hi.y, hi.z, c.y * theta);
        const float wi = a.wsum_inv[i];
        const float ws = a.w_const * (float)s.alive;
        a.damage[i] = wi > 0.0f ? fmaxf(0.0f, 1.0f - ws * wi) : 0.0f;
    }
}

// the force loop and the node's update (FP32 force, FP64 u, as the bond step);
// its walk in pairs of bonds wants 80 registers (3 resident blocks per SM)
__global__ void __launch_bounds__(PD_LAT_THREADS, 3)
    k_osb_lat_force(const __grid_constant__ StepArgsF32 a, const OsbLatArgs o)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = lat_step_of(a);
    lat_advance_counter(a);  // the step's last kernel
    const int cur = (int)(step & 1);
    const int64_t nslices = (a.n + 31) >> 5;
    float4* __restrict__ Pout = const_cast<float4*>(a.lat_pub[cur ^ 1]);
    const double* __restrict__ U = a.lat_u[cur];
    double* __restrict__ Uout = a.lat_u[cur ^ 1];
    const float4* __restrict__ S = o.rec;
    for (int64_t g = wid; g < nslices; g += nwarps) {
        OsbForceNode s;
        s.i = (g << 5) + lane;
        const float4 r0 = ld_pub(S + s.i);
        s.nx = make_float2(-r0.x, -r0.x);
        s.ny = make_float2(-r0.y, -r0.y);
        s.nz = make_float2(-r0.z, -r0.z);
        s.A = r0.w;
        s.B = o.bco[s.i];
        const uint32_t* bw = a.bits + g * 4 * 32 + lane;
#pragma unroll
        for (int q = 0; q < 4; ++q) s.word[q] = bw[q * 32];
        s.fx = s.fy = s.fz = make_float2(0.f, 0.f);
        if (o.exact[g]) {  // a bond of the slice has |x| past the series (or is near s_c)
            s.own.nxy = make_float2(-r0.x, -r0.y);
            s.own.nz = -r0.z;
            s.fxy = make_float2(0.f, 0.f);
            s.fzs = 0.f;
            osb_force_walk(a, S + s.i, o.bco + s.i, s,
                           std::make_integer_sequence<int, kStencilSegs>{});
            s.fx.x = s.fxy.x;
            s.fy.x = s.fxy.y;
            s.fz.x = s.fzs;
        } else {
            osb_force_pairwalk(a, S + s.i, o.bco + s.i, s,
                               std::make_integer_sequence<int, kStencilSegs>{});
        }
        const int64_t i = s.i;
        if (i >= a.n) continue;
        const float V = a.w_const;  // the volume (uniform)
        const uint32_t cls = a.bcc[i];
        uint32_t mask = 0u;
        const BcClass* bc = nullptr;
        float F[3] = {V * (s.fx.x + s.fx.y), V * (s.fy.x + s.fy.y), V * (s.fz.x + s.fz.y)};
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
                                int grid_force, int block, cudaStream_t s)
{
    if (sc_mode == 0)
        k_osb_lat_dilation<0><<<grid, block, 0, s>>>(a, o);
    else
        k_osb_lat_dilation<1><<<grid, block, 0, s>>>(a, o);
    if (cudaPeekAtLastError() == cudaSuccess) k_osb_lat_force<<<grid_force, block, 0, s>>>(a, o);
    return cudaGetLastError();
}

}  // namespace pd
