// FP32-bulk step of a model on a regular cubic lattice: the stencil kernel.
//
// The fused step of k_step_f32 (Eqs. 4-6, 10-11, damped Euler-Cromer,
// displacement BCs, damage of Eq. 8) for the common case of the paper's
// benchmark bodies: nodes on a cubic lattice of spacing dx with
// 3 dx <= delta < sqrt(10) dx, so that every family is a subset of the 122
// stencil offsets (see stencil_offset).  Such a model is stored in lattice
// order p = (ix Ny + iy) Nz + iz with slot m of every node's flags holding
// stencil offset m.  The neighbour across offset o is then node p + o_x Sx +
// o_y Sy + o_z, and the reference bond is xi = kappa o in horizon units
// (kappa = dx / delta), both fixed when the kernel is compiled up to the two
// strides and kappa, which come in as kernel parameters:
//   - no neighbour ids are read (the family is implicit in the lattice; the
//     flags say which offsets are bonds: absent members, bonds cut by a notch
//     and broken bonds all have flag 0),
//   - no positions are read or subtracted, |xi|^2 and |xi| are constants of
//     the offset, and the offsets' zero components drop out of the arithmetic,
//   - the slot loop is unrolled over the stencil at compile time: flag bits,
//     record offsets along z (immediates) and per-offset constants are fixed.
// A lane owns one node and accumulates its force in registers; a warp walks 32
// consecutive nodes.  The walk takes the stencil's bonds two at a time (two
// rows of a segment at the same position, or o_z and -o_z of the o_x = o_y = 0
// row: the same |xi|), each quantity of the two bonds in one register pair
// through paired FP32 instructions.  Where the 32 nodes cross a lattice line the offsets of
// some lanes wrap to other nodes; those slots have flag 0 and are masked, and
// the published records carry a zero halo so that every read stays in bounds.
//
// Precision (the FP32-bulk reading): each node's displacement is accumulated
// in FP64 (u / delta, double buffered) and published to the neighbours rounded
// to FP32, 16 bytes per node.  The bulk bond arithmetic is FP32 on those
// published values; the rounding of u/delta to FP32 acts on the forces as a
// displacement perturbation of at most half an ulp of |u|, drawn anew at every
// step, so it does not accumulate.  Bonds whose FP32 stretch reaches a band
// just below the smallest s_c are decided from the FP64 displacements: in FP32
// away from the bond's s_c and with the literal FP64 stretch of Eq. 4 near it.
//
// Per bond (offset o, q = |o|^2, L = |xi|):
//   eta = h_j - h_i                       published displacements / delta
//   y   = xi + eta,   num = eta . (2 xi + eta) = |y|^2 - L^2 (no cancellation)
//   |y| = y2 rsqrt(y2) with y2 = L^2 + num
//   D   = L^2 |y| + L y2 = den |y|,  den = L (L + |y|),  s = num / den
//   f   = w s y / |y| = w (num / D) y
// The band test runs on num: s >= fast_lo <=> |y| >= L (1 + fast_lo) <=>
// num >= fast_lo (2 + fast_lo) L^2, a per-q threshold; candidates are decided
// after each flag word.  Both directions of a bond do the same operations on
// negated inputs, so their forces are exact negatives and they break together.
//
// Batch build (pd_step_f32_lat_batch.cu, PD_LAT_BATCH): many lattice models in
// one launch, each instance's state in units of its own spacing (kappa = 1, so
// the stencil's constants are the same for all), its strides, near-s_c
// threshold and material taken per node from the instance table.
#define PD_F32_LAT 1
#include "pd_step_f32.cu"

#include <utility>

#ifndef PD_LAT_BATCH
#define PD_LAT_BATCH 0
#endif
// Helper builds (the state-based loops, pd_step_f32_lat_osb.cu, and the
// shared-memory tile step, pd_step_f32_lat_tma.cu): this file's helpers without
// the bond-based step's entry points.
#ifndef PD_LAT_HELPERS
#define PD_LAT_HELPERS 0
#endif

namespace pd {
namespace {

constexpr bool kLatBatch = PD_LAT_BATCH != 0;

#ifndef PD_LAT_THREADS
#define PD_LAT_THREADS 256
#endif
// resident blocks of 256 threads per SM the register allocation is made for:
// 4 (64 registers, the default) or 3 (80 registers, pd_step_f32_lat_r80.cu);
// pd_autotune times both
#ifndef PD_LAT_MIN_BLOCKS
#define PD_LAT_MIN_BLOCKS 4
#endif

// the stencil offsets for run-time slot numbers (near-s_c resolution)
struct StencilTab {
    signed char o[kStencilSlots][4];
};
constexpr StencilTab make_stencil_tab()
{
    StencilTab t{};
    for (int m = 0; m < kStencilSlots; ++m) {
        const Off3 o = stencil_offset(m);
        t.o[m][0] = (signed char)o.x;
        t.o[m][1] = (signed char)o.y;
        t.o[m][2] = (signed char)o.z;
        t.o[m][3] = (signed char)o.q;
    }
    return t;
}
__constant__ StencilTab c_stencil = make_stencil_tab();

__device__ __forceinline__ float rsqrt_fast(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_fast(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// one published record (16 bytes) with a single 128-bit non-coherent load
__device__ __forceinline__ float4 ld_pub(const float4* p)
{
    float4 r;
    asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}

// The lane's own published displacement, negated: (x, y) as one register pair
struct LatOwn {
    float2 nxy;
    float nz;
};

__device__ __forceinline__ float3 lat_eta(const LatOwn& i, const float4 j)
{
    const float2 d = __fadd2_rn(make_float2(j.x, j.y), i.nxy);
    return make_float3(d.x, d.y, j.z + i.nz);
}

// The break decision of the bond i -> j (offset (ox, oy, oz), q = |o|^2) whose
// FP32 stretch reached the near-s_c band, from the FP64 displacements: in FP32
// away from the bond's s_c, with the literal FP64 stretch of Eq. 4 near it; then
// the no-fail rule.
__device__ __forceinline__ bool lat_breaks(const StepArgsF32& a, int cur, int64_t i, int64_t j,
                                           int ox, int oy, int oz, int q, double sc_single)
{
    const double* __restrict__ U = a.lat_u[cur];
    double e64[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) e64[c] = U[3 * j + c] - U[3 * i + c];
    // FP32 stretch terms from the FP64 displacement difference
    const float xx = a.lat_xi[ox + 3], xy = a.lat_xi[oy + 3], xz = a.lat_xi[oz + 3];
    const float ex = (float)e64[0], ey = (float)e64[1], ez = (float)e64[2];
    const float num = fmaf(ex, ex + 2.0f * xx, fmaf(ey, ey + 2.0f * xy, ez * (ez + 2.0f * xz)));
    const float y2 = num + a.lat_q[q];
    const float ay = y2 * rsqrt_fast(y2);
    const float D = fmaf(ay, a.lat_q[q], a.lat_l[q] * y2);
    double sc = sc_single;
    double unit = a.delta;
    if (kLatBatch) {  // the instance's own s_c (local ids as keys) and length unit
        const InstParams& ip = a.itab[a.inst[i]];
        sc = ip.sc_mode == 1 ? sc_draw(ip.sc_seed, ip.sc_lo, ip.sc_hi, a.hid[i], a.hid[j]) : ip.sc;
        unit = ip.unit;
    }
    const float scf = (float)sc;
    // num |y| - s_c D = den |y| (s - s_c): its sign decides, away from s_c
    const float r = fmaf(-scf, D, num * ay);
    bool brk;
    if (fabsf(r) > a.guard * scf * D) {
        brk = r >= 0.0f;
    } else {
        double xv[3], y[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xv[c] = a.x64[3 * j + c] - a.x64[3 * i + c];
            y[c] = xv[c] + e64[c] * unit;
        }
        const double L = sqrt(xv[0] * xv[0] + xv[1] * xv[1] + xv[2] * xv[2]);
        const double Rr = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
        brk = (Rr - L) / L >= sc;
    }
    if (brk && a.has_nofail) brk = ((a.bct[a.bcc[i]].mask | a.bct[a.bcc[j]].mask) & 8u) == 0u;
    return brk;
}

// A candidate bond of slot m (its stretch in the near-s_c band, or |x| past the
// walk's series): the break decision (lat_breaks) and the correction of the
// force term the walk added for it: minus that term when the bond breaks, the
// exact term (num / D) minus the series one when |x| > kLatPolyX, else zero.
// slot: the bond's index in the per-slot arrays; sx, sy: a batch instance's
// strides.
template <int SCM, bool PBC>
__device__ __noinline__ float3 lat_resolve(const StepArgsF32& a, int cur, int64_t i, int m,
                                           int64_t slot, int sx, int sy, bool* broken)
{
    const int ox = c_stencil.o[m][0], oy = c_stencil.o[m][1], oz = c_stencil.o[m][2];
    const int q = c_stencil.o[m][3];
    if (!kLatBatch) {  // a single model: its strides are kernel parameters
        sx = a.lat_sx;
        sy = a.lat_sy;
    }
    const int64_t j = i + (int64_t)ox * sx + (int64_t)oy * sy + oz;
    const double sc = SCM == 1 ? sc_draw(a.sc_seed, a.sc_lo, a.sc_hi, a.gid[i], a.gid[j]) : a.sc;
    const bool brk = lat_breaks(a, cur, i, j, ox, oy, oz, q, sc);
    *broken = brk;
    // the walk's force term from the published displacements, formed as it formed it
    const float xx = a.lat_xi[ox + 3], xy = a.lat_xi[oy + 3], xz = a.lat_xi[oz + 3];
    const float4* __restrict__ P = a.lat_pub[cur];
    const float4 hi = ld_pub(P + i), hj = ld_pub(P + j);
    LatOwn own;
    own.nxy = make_float2(-hi.x, -hi.y);
    own.nz = -hi.z;
    const float3 e = lat_eta(own, hj);
    const float fx = e.x + xx, fy = e.y + xy, fz = e.z + xz;
    const float n2 = fmaf(e.x, e.x + 2.0f * xx, fmaf(e.y, e.y + 2.0f * xy, e.z * (e.z + 2.0f * xz)));
    const float cs = n2 * fmaf(fmaf(a.lat_pc[2][q], n2, a.lat_pc[1][q]), n2, a.lat_pc[0][q]);
    float dc;
    if (brk) {
        dc = -cs;
    } else if (fabsf(n2) > a.lat_pt[q]) {  // past the series' range: the exact num / D
        const float z2 = n2 + a.lat_q[q];
        const float az = z2 * rsqrt_fast(z2);
        const float Dz = fmaf(az, a.lat_q[q], a.lat_l[q] * z2);
        dc = n2 * rcp_fast(Dz) - cs;
    } else {
        return make_float3(0.f, 0.f, 0.f);
    }
    if (PBC) dc *= a.cbond[slot];
    return make_float3(dc * fx, dc * fy, dc * fz);
}

// The step a launch computes: the device counter plus the launch's offset, or
// the absolute step of a direct launch (a.step_abs >= 0), whose kernel then sets
// the counter to the next step itself (block 0, thread 0: no thread of such a
// launch reads it, and the stream orders it before the next launch)
__device__ __forceinline__ int64_t lat_step_of(const StepArgsF32& a)
{
    return a.step_abs >= 0 ? a.step_abs : a.step_ctr[0] + a.k;
}
__device__ __forceinline__ void lat_advance_counter(const StepArgsF32& a)
{
    if (a.step_abs >= 0 && blockIdx.x == 0 && threadIdx.x == 0)
        const_cast<int64_t*>(a.step_ctr)[0] = a.step_abs + 1;
}

// One node's state over its stencil walk.  The walk takes its bonds two at a
// time (lat_pair_bond): the first half of each register pair belongs to the
// first bond of a pair, the second half to the second.
struct LatNode {
    float2 nx, ny, nz;  // the lane's own published displacement, negated, twice
    int sx, sy;         // batch: the instance's node-order strides
    float cc_t, ch_t;   // batch: its candidate test per unit q
    int64_t i;
    int64_t slot0;      // index of slot 0 of this node in per-slot arrays
    float2 fx, fy, fz;  // force sums over the first and the second bonds of the pairs
    uint32_t word[4];   // bond flags (stencil slot order)
    uint32_t pend;      // near-s_c candidates of the current flag word
    int alive;          // intact bonds after this step's decisions
};

// start of a node's walk from its own published record
__device__ __forceinline__ void lat_node_begin(LatNode& s, const float4 hi)
{
    s.nx = make_float2(-hi.x, -hi.x);
    s.ny = make_float2(-hi.y, -hi.y);
    s.nz = make_float2(-hi.z, -hi.z);
    s.fx = make_float2(0.f, 0.f);
    s.fy = make_float2(0.f, 0.f);
    s.fz = make_float2(0.f, 0.f);
    s.pend = 0u;
    s.alive = 0;
}

// Where the walk reads the neighbours' published records.  SrcGlobal: the
// record array itself (a row of offsets o_x, o_y starts o_x Sx + o_y Sy records
// from the node's own); SrcTile: a shared-memory copy of the records of a box of
// the lattice, z fastest, TZ x TY records per x plane (a row starts
// TZ (o_y + TY o_x) records from the node's own).
struct SrcGlobal {
    __device__ static int64_t fixed_row(const StepArgsF32& a, const LatNode& s, int ox, int oy)
    {
        return kLatBatch ? (int64_t)(ox * s.sx + oy * s.sy) : (int64_t)(ox * a.lat_sx + oy * a.lat_sy);
    }
    __device__ static int64_t loop_row(const StepArgsF32& a, const LatNode& s, int r)
    {
        return kLatBatch ? (int64_t)(a.lat_rox[r] * s.sx + a.lat_roy[r] * s.sy)
                         : (int64_t)a.lat_roff[r];
    }
    __device__ static float4 load(const float4* p) { return ld_pub(p); }
};

template <int TZ, int TY>
struct SrcTile {
    __device__ static int fixed_row(const StepArgsF32&, const LatNode&, int ox, int oy)
    {
        return TZ * (oy + TY * ox);
    }
    __device__ static int loop_row(const StepArgsF32& a, const LatNode&, int r)
    {
        return TZ * (a.lat_roy[r] + TY * a.lat_rox[r]);
    }
    __device__ static float4 load(const float4* p) { return *p; }
};

// Two bonds of equal |xi| walked together: bond K0 of the row at P0 (flags
// from bit 0 in rb0, candidates into rp0) and bond K1 of the row at P1 (rb1,
// rp1), both rows with q_xy = QXY: two rows of one segment at the same
// position, or mirror positions of the o_x = o_y = 0 row.  xix, xiy, xi2x,
// xi2y: the two rows' x and y components of xi and 2 xi (ZX / ZY: 0 in both).
// Every quantity of the two bonds sits in one register pair and goes through
// paired FP32 instructions, each half rounded as the scalar operation, so each
// bond's terms are those of the one-bond formulas (lat_resolve re-forms them).
template <class Src, int QXY, int K0, int K1, int ZX, int ZY, bool PBC>
__device__ __forceinline__ void lat_pair_bond(const StepArgsF32& a, const float2 xix,
                                              const float2 xiy, const float2 xi2x,
                                              const float2 xi2y, const float4* P0,
                                              const float4* P1, const float* cb0,
                                              const float* cb1, uint32_t rb0, uint32_t rb1,
                                              uint32_t& rp0, uint32_t& rp1, LatNode& s)
{
    constexpr int OZ0 = stencil_row_oz(QXY, K0), OZ1 = stencil_row_oz(QXY, K1);
    static_assert(OZ0 * OZ0 == OZ1 * OZ1, "the two bonds of a pair have the same |xi|");
    constexpr int Q = QXY + OZ0 * OZ0;
    const float4 r0 = Src::load(P0 + OZ0), r1 = Src::load(P1 + OZ1);
    const float2 ex = __fadd2_rn(make_float2(r0.x, r1.x), s.nx);
    const float2 ey = __fadd2_rn(make_float2(r0.y, r1.y), s.ny);
    const float2 ez = __fadd2_rn(make_float2(r0.z, r1.z), s.nz);
    const float2 yx = ZX ? ex : __fadd2_rn(ex, xix);
    const float2 tx = ZX ? ex : __fadd2_rn(ex, xi2x);
    const float2 yy = ZY ? ey : __fadd2_rn(ey, xiy);
    const float2 ty = ZY ? ey : __fadd2_rn(ey, xi2y);
    const float2 yz = OZ0 ? __fadd2_rn(ez, make_float2(a.lat_xi[OZ0 + 3], a.lat_xi[OZ1 + 3])) : ez;
    const float2 tz = OZ0 ? __fadd2_rn(ez, make_float2(a.lat_xi2[OZ0 + 3], a.lat_xi2[OZ1 + 3]))
                          : ez;
    // num = eta . (2 xi + eta); an absent or broken bond (flag 0) has num = 0: no
    // force and no candidate
    float2 num = __ffma2_rn(ex, tx, __ffma2_rn(ey, ty, __fmul2_rn(ez, tz)));
    num.x = ((rb0 >> K0) & 1u) ? num.x : 0.0f;
    num.y = ((rb1 >> K1) & 1u) ? num.y : 0.0f;
    // coefficient num / D = num g(x) / |xi|^3, x = num / |xi|^2, g(x) = 1 / (r (1 + r))
    // with r = sqrt(1 + x): the series of g to x^2 (1/2 - 3x/8 + 5x^2/16), within
    // 0.25 ulp for |x| <= kLatPolyX, in place of a square root and a division
    float2 coef = __fmul2_rn(
        num, __ffma2_rn(__ffma2_rn(a.lat_pcd[2][Q], num, a.lat_pcd[1][Q]), num, a.lat_pcd[0][Q]));
    if (PBC) {
        coef.x *= __ldg(cb0 + 32 * K0);
        coef.y *= __ldg(cb1 + 32 * K1);
    }
    // candidates: the near-s_c band and |x| past the series (num >= min(thr, pt)
    // or num <= -pt), decided and corrected after the flag word (lat_word_end);
    // they keep the series term here
    if (kLatBatch) {
        const float ch = (float)Q * s.ch_t;
        rp0 |= fabsf(fmaf(-(float)Q, s.cc_t, num.x)) >= ch ? (1u << K0) : 0u;
        rp1 |= fabsf(fmaf(-(float)Q, s.cc_t, num.y)) >= ch ? (1u << K1) : 0u;
    } else {
        const float2 d = __fadd2_rn(num, a.lat_ccd[Q]);
        rp0 |= fabsf(d.x) >= a.lat_ch[Q] ? (1u << K0) : 0u;
        rp1 |= fabsf(d.y) >= a.lat_ch[Q] ? (1u << K1) : 0u;
    }
    s.fx = __ffma2_rn(coef, yx, s.fx);
    s.fy = __ffma2_rn(coef, yy, s.fy);
    s.fz = __ffma2_rn(coef, yz, s.fz);
}

// Rows R and R + 1 (compile-time) of segment SG, unrolled, their offsets fixed
template <class Src, bool PBC, int SG, int R, int... K>
__device__ __forceinline__ void lat_rowpair_fixed(const StepArgsF32& a, const float4* Pi,
                                                  LatNode& s, std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    constexpr Off3 o0 = stencil_row_xy(sg.qxy, sg.row0 + R);
    constexpr Off3 o1 = stencil_row_xy(sg.qxy, sg.row0 + R + 1);
    constexpr int b0 = sg.bit0 + len * R;
    const float4* P0 = Pi + Src::fixed_row(a, s, o0.x, o0.y);
    const float4* P1 = Pi + Src::fixed_row(a, s, o1.x, o1.y);
    const uint32_t rb0 = s.word[sg.word] >> b0, rb1 = rb0 >> len;
    const float* cb0 = PBC ? a.cbond + s.slot0 + 32 * (32 * sg.word + b0) : nullptr;
    const float* cb1 = PBC ? cb0 + 32 * len : nullptr;
    uint32_t rp0 = 0u, rp1 = 0u;
    const float2 xix = make_float2(a.lat_xi[o0.x + 3], a.lat_xi[o1.x + 3]);
    const float2 xiy = make_float2(a.lat_xi[o0.y + 3], a.lat_xi[o1.y + 3]);
    const float2 xi2x = make_float2(a.lat_xi2[o0.x + 3], a.lat_xi2[o1.x + 3]);
    const float2 xi2y = make_float2(a.lat_xi2[o0.y + 3], a.lat_xi2[o1.y + 3]);
    (lat_pair_bond<Src, sg.qxy, K, K, o0.x == 0 && o1.x == 0, o0.y == 0 && o1.y == 0, PBC>(
         a, xix, xiy, xi2x, xi2y, P0, P1, cb0, cb1, rb0, rb1, rp0, rp1, s),
     ...);
    s.pend |= (rp0 | (rp1 << len)) << b0;
}

template <class Src, bool PBC, int SG, int... R>
__device__ __forceinline__ void lat_rows_fixed(const StepArgsF32& a, const float4* Pi, LatNode& s,
                                               std::integer_sequence<int, R...>)
{
    (lat_rowpair_fixed<Src, PBC, SG, 2 * R>(
         a, Pi, s, std::make_integer_sequence<int, stencil_row_len(stencil_seg(SG).qxy)>{}),
     ...);
}

// The o_x = o_y = 0 row (a segment of one row, o_z = -3..-1, 1..3): its
// positions K and len - 1 - K (o_z and -o_z) as pairs
template <class Src, bool PBC, int SG, int... K>
__device__ __forceinline__ void lat_row_mirror(const StepArgsF32& a, const float4* Pi, LatNode& s,
                                               std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    static_assert(sg.qxy == 0 && sg.nrows == 1 && len % 2 == 0, "the o_x = o_y = 0 row");
    const uint32_t rb = s.word[sg.word] >> sg.bit0;
    const float* cb = PBC ? a.cbond + s.slot0 + 32 * (32 * sg.word + sg.bit0) : nullptr;
    uint32_t rp = 0u;
    const float2 z = make_float2(0.f, 0.f);
    (lat_pair_bond<Src, sg.qxy, K, len - 1 - K, 1, 1, PBC>(a, z, z, z, z, Pi, Pi, cb, cb, rb, rb,
                                                          rp, rp, s),
     ...);
    s.pend |= rp << sg.bit0;
}

// Segment SG as a loop over its rows, two rows per iteration (offsets of a row
// unrolled)
template <class Src, bool PBC, int SG, int... K>
__device__ __forceinline__ void lat_rows_loop(const StepArgsF32& a, const float4* Pi, LatNode& s,
                                              std::integer_sequence<int, K...>)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    static_assert(sg.nrows % 2 == 0, "a loop segment walks its rows in pairs");
#pragma unroll 1
    for (int r = 0; r < sg.nrows; r += 2) {
        const int j = sg.first + r;
        const float4 xa = a.lat_rxp[j][0], xb = a.lat_rxp[j][1];
        const float4* P0 = Pi + Src::loop_row(a, s, j);
        const float4* P1 = Pi + Src::loop_row(a, s, j + 1);
        const int b0 = sg.bit0 + len * r;
        const uint32_t rb0 = s.word[sg.word] >> b0, rb1 = rb0 >> len;
        const float* cb0 = PBC ? a.cbond + s.slot0 + 32 * (32 * sg.word + b0) : nullptr;
        const float* cb1 = PBC ? cb0 + 32 * len : nullptr;
        uint32_t rp0 = 0u, rp1 = 0u;
        (lat_pair_bond<Src, sg.qxy, K, K, sg.zx, sg.zy, PBC>(
             a, make_float2(xa.x, xa.y), make_float2(xa.z, xa.w), make_float2(xb.x, xb.y),
             make_float2(xb.z, xb.w), P0, P1, cb0, cb1, rb0, rb1, rp0, rp1, s),
         ...);
        s.pend |= (rp0 | (rp1 << len)) << b0;
    }
}

template <class Src, bool PBC, int SG>
__device__ __forceinline__ void lat_seg(const StepArgsF32& a, const float4* Pi, LatNode& s)
{
    constexpr StencilSeg sg = stencil_seg(SG);
    constexpr int len = stencil_row_len(sg.qxy);
    if constexpr (!sg.unroll)
        lat_rows_loop<Src, PBC, SG>(a, Pi, s, std::make_integer_sequence<int, len>{});
    else if constexpr (sg.nrows == 1)
        lat_row_mirror<Src, PBC, SG>(a, Pi, s, std::make_integer_sequence<int, len / 2>{});
    else
        lat_rows_fixed<Src, PBC, SG>(a, Pi, s, std::make_integer_sequence<int, sg.nrows / 2>{});
}

// After the last segment of flag word W: decide the word's near-s_c candidates.
template <int SCM, bool PBC, int W>
__device__ __forceinline__ void lat_word_end(const StepArgsF32& a, int cur, LatNode& s)
{
    uint32_t nword = s.word[W];
    uint32_t pend = s.pend;
    while (pend) {
        const int bb = __ffs(pend) - 1;
        pend &= pend - 1u;
        bool broken;
        const int m = 32 * W + bb;
        const float3 f = lat_resolve<SCM, PBC>(a, cur, s.i, m, s.slot0 + 32 * m,
                                               kLatBatch ? s.sx : 0, kLatBatch ? s.sy : 0,
                                               &broken);
        if (broken) nword &= ~(1u << bb);
        s.fx.x += f.x;  // the candidate's correction (lat_resolve)
        s.fy.x += f.y;
        s.fz.x += f.z;
    }
    s.word[W] = nword;
    s.alive += __popc(nword);
    s.pend = 0u;
}

// the walk over the stencil: the segments of each flag word, then the word's
// near-s_c candidates (the segment and word layout of stencil_seg)
template <class Src, int SCM, bool PBC>
__device__ __forceinline__ void lat_walk(const StepArgsF32& a, int cur, const float4* Pi,
                                         LatNode& s)
{
    lat_seg<Src, PBC, 0>(a, Pi, s);
    lat_seg<Src, PBC, 1>(a, Pi, s);
    lat_seg<Src, PBC, 2>(a, Pi, s);
    lat_word_end<SCM, PBC, 0>(a, cur, s);
    lat_seg<Src, PBC, 3>(a, Pi, s);
    lat_seg<Src, PBC, 4>(a, Pi, s);
    lat_seg<Src, PBC, 5>(a, Pi, s);
    lat_word_end<SCM, PBC, 1>(a, cur, s);
    lat_seg<Src, PBC, 6>(a, Pi, s);
    lat_seg<Src, PBC, 7>(a, Pi, s);
    lat_seg<Src, PBC, 8>(a, Pi, s);
    lat_word_end<SCM, PBC, 2>(a, cur, s);
    lat_seg<Src, PBC, 9>(a, Pi, s);
    lat_word_end<SCM, PBC, 3>(a, cur, s);
}
static_assert(stencil_seg(2).word == 0 && stencil_seg(3).word == 1 && stencil_seg(5).word == 1 &&
                  stencil_seg(6).word == 2 && stencil_seg(8).word == 2 && stencil_seg(9).word == 3,
              "lat_walk follows the segment layout");

// The node's update: damped Euler-Cromer (Eq. 11) with the force in FP32 and
// u accumulated in FP64, the linear displacement ramp, damage (Eq. 8) from the
// intact-bond count; publishes the FP32 rounding of the new u / delta.
__device__ __forceinline__ void lat_update(const StepArgsF32& a, const LatNode& s, int64_t step,
                                           const double* __restrict__ U,
                                           double* __restrict__ Uout, float4* __restrict__ Pout)
{
    const int64_t i = s.i;
    float wc = a.w_const, dtd = a.dtd_f;
    double inv_unit = a.inv_delta;
    if (kLatBatch) {
        const InstParams& ip = a.itab[a.inst[i]];
        wc = ip.w_const;
        dtd = ip.dtd;
        inv_unit = ip.inv_unit;
    }
    const uint32_t cls = a.bcc[i];
    uint32_t mask = 0u;
    const BcClass* bc = nullptr;
    float F[3] = {wc * (s.fx.x + s.fx.y), wc * (s.fy.x + s.fy.y), wc * (s.fz.x + s.fz.y)};
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
        un[c] = fma((double)vn, (double)dtd, U[3 * i + c]);
        if (mask & (1u << c)) {
            const double s_now = a.disp_rate * (double)step;
            const double s_next = a.disp_rate * (double)(step + 1);
            un[c] = bc->disp[c] * s_next * inv_unit;
            vn = (float)(bc->disp[c] * (s_next - s_now) / a.dt);
        }
        finite = finite && isfinite(un[c]);
        a.v[3 * i + c] = vn;
        Uout[3 * i + c] = un[c];
    }
    Pout[i] = make_float4((float)un[0], (float)un[1], (float)un[2], 0.0f);
    const float wi = a.wsum_inv[i];
    const float ws = wc * (float)s.alive;
    a.damage[i] = wi > 0.0f ? fmaxf(0.0f, 1.0f - ws * wi) : 0.0f;
    if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
}

template <int SCM, bool PBC>
__global__ void __launch_bounds__(PD_LAT_THREADS, PD_LAT_MIN_BLOCKS)
    k_step_f32_lat(const __grid_constant__ StepArgsF32 a)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = lat_step_of(a);
    lat_advance_counter(a);
    const int cur = (int)(step & 1);
    const int64_t nslices = (a.n + 31) >> 5;
    const float4* __restrict__ P = a.lat_pub[cur];
    float4* __restrict__ Pout = const_cast<float4*>(a.lat_pub[cur ^ 1]);
    const double* __restrict__ U = a.lat_u[cur];
    double* __restrict__ Uout = a.lat_u[cur ^ 1];

    for (int64_t g = wid; g < nslices; g += nwarps) {
        LatNode s;
        s.i = (g << 5) + lane;
        s.slot0 = g * 128 * 32 + lane;
        if (kLatBatch) {
            const InstParams& ip = a.itab[a.inst[s.i]];
            s.sx = ip.lat_sx;
            s.sy = ip.lat_sy;
            s.cc_t = ip.lat_cc_t;
            s.ch_t = ip.lat_ch_t;
        }
        lat_node_begin(s, ld_pub(P + s.i));
        uint32_t* bw = a.bits + g * 4 * 32 + lane;
        uint32_t w0[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) w0[q] = s.word[q] = bw[q * 32];
        lat_walk<SrcGlobal, SCM, PBC>(a, cur, P + s.i, s);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (s.word[q] != w0[q]) bw[q * 32] = s.word[q];

        if (s.i >= a.n) continue;
        lat_update(a, s, step, U, Uout, Pout);
    }
}

}  // namespace

#if !PD_LAT_HELPERS
// entry points of this build: single model or batch, register budget
#if PD_LAT_BATCH && PD_LAT_MIN_BLOCKS == 3
#define PD_LAT_KERNEL_OF step_f32_kernel_lat_batch_r80
#define PD_LAT_LAUNCH launch_step_f32_lat_batch_r80
#elif PD_LAT_BATCH
#define PD_LAT_KERNEL_OF step_f32_kernel_lat_batch
#define PD_LAT_LAUNCH launch_step_f32_lat_batch
#elif PD_LAT_MIN_BLOCKS == 3
#define PD_LAT_KERNEL_OF step_f32_kernel_lat_r80
#define PD_LAT_LAUNCH launch_step_f32_lat_r80
#else
#define PD_LAT_KERNEL_OF step_f32_kernel_lat
#define PD_LAT_LAUNCH launch_step_f32_lat
#endif

const void* PD_LAT_KERNEL_OF(int sc_mode, bool per_bond_c)
{
    if (per_bond_c)
        return sc_mode == 0 ? (const void*)k_step_f32_lat<0, true> : (const void*)k_step_f32_lat<1, true>;
    return sc_mode == 0 ? (const void*)k_step_f32_lat<0, false> : (const void*)k_step_f32_lat<1, false>;
}

cudaError_t PD_LAT_LAUNCH(const StepArgsF32& a, int sc_mode, int grid, int block, cudaStream_t s)
{
    const bool pbc = a.cbond != nullptr;
    if (sc_mode == 0) {
        if (pbc) k_step_f32_lat<0, true><<<grid, block, 0, s>>>(a);
        else k_step_f32_lat<0, false><<<grid, block, 0, s>>>(a);
    } else {
        if (pbc) k_step_f32_lat<1, true><<<grid, block, 0, s>>>(a);
        else k_step_f32_lat<1, false><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}
#endif  // !PD_LAT_HELPERS

}  // namespace pd
