// FP32-bulk step of a model on a regular cubic lattice: the stencil kernel.
//
// The same fused step as k_step_f32 (Eqs. 4-6, 10-11, damped Euler-Cromer,
// displacement BCs, damage of Eq. 8) for the common case of the paper's
// benchmark bodies: nodes on a cubic lattice of spacing dx with
// 3 dx <= delta < sqrt(10) dx, so that every family is a subset of the 122
// stencil offsets (see stencil_offset).  Such a model is stored in lattice
// order p = (ix Ny + iy) Nz + iz with slot m of every node's flags holding
// stencil offset m.  The neighbour across offset o is then node p + o_x Sx +
// o_y Sy + o_z, and the reference bond is xi = kappa o in horizon units
// (kappa = dx / delta), both known when the kernel is compiled up to the two
// strides and kappa, which come in as kernel parameters:
//   - no neighbour ids are read (the family is implicit in the lattice; the
//     flags say which offsets are bonds: absent members, bonds cut by a notch
//     and broken bonds all have flag 0),
//   - no positions are read or subtracted, |xi|^2 and |xi| are constants of
//     the offset, and the offsets' zero components drop out of the arithmetic,
//   - the slot loop is unrolled over the stencil at compile time: flag bits,
//     record offsets along z (immediates) and per-offset constants are fixed.
// A lane still owns one node and accumulates its force in registers; a warp
// walks 32 consecutive nodes.  Where the 32 nodes cross a lattice line the
// offsets of some lanes wrap to other nodes; those slots have flag 0 and are
// masked, and the node records carry a zero halo so that every read stays in
// bounds.
//
// Per bond (offset o, q = |o|^2, L = |xi|):
//   eta = (h_j - h_i) + (l_j - l_i)       published float-float displacement
//   y   = xi + eta,   num = eta . (2 xi + eta) = |y|^2 - L^2 (no cancellation)
//   |y| = y2 rsqrt(y2) with y2 = L^2 + num
//   D   = L^2 |y| + L y2 = den |y|,  den = L (L + |y|),  s = num / den
//   f   = w s y / |y| = w (num / D) y
// The break test runs on num: s >= fast_lo <=> |y| >= L (1 + fast_lo) <=>
// num >= fast_lo (2 + fast_lo) L^2, a per-q threshold.  Such bonds (near the
// smallest s_c) are decided after each flag word, as in k_step_f32: in FP32
// away from the bond's s_c and with the literal FP64 stretch of Eq. 4 within a
// relative band of it.  Both directions of a bond do the same operations on
// negated inputs, so their forces are exact negatives and they break together.
#define PD_F32_LAT 1
#include "pd_step_f32.cu"

#include <utility>

namespace pd {
namespace {

// the stencil offsets for run-time slot numbers (near-s_c resolution)
struct StencilTab {
    signed char o[kStencil][4];
};
constexpr StencilTab make_stencil_tab()
{
    StencilTab t{};
    for (int m = 0; m < kStencil; ++m) {
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

// The lane's own record as the bond terms subtract it: negated register pairs
// (z, h_x), (h_y, h_z), (l_x, l_z) of the 256-bit load, and l_y.
struct LatOwn {
    float2 zhx, hyz, lxz;
    float ly;
};

__device__ __forceinline__ LatOwn lat_own(const float4 a, const float4 b)
{
    LatOwn p;
    p.zhx = make_float2(-a.z, -a.w);
    p.hyz = make_float2(-b.x, -b.y);
    p.lxz = make_float2(-b.z, -b.w);
    p.ly = -bf_lo(b.z);
    return p;
}

// eta = u_j - u_i / delta from the published float-float displacements
__device__ __forceinline__ float3 lat_eta(const LatOwn& i, const float4 ja, const float4 jb)
{
    const float2 d1 = __fadd2_rn(make_float2(ja.z, ja.w), i.zhx);  // (., dh_x)
    const float2 d2 = __fadd2_rn(make_float2(jb.x, jb.y), i.hyz);  // (dh_y, dh_z)
    const float2 d3 = __fadd2_rn(make_float2(jb.z, jb.w), i.lxz);  // (dl_x, dl_z)
    const float dly = bf_lo(jb.z) + i.ly;
    return make_float3(d1.y + d3.x, d2.x + dly, d2.y + d3.y);
}

// Bond terms of offset o = (OX, OY, OZ), q = |o|^2, from eta: y, num,
// D = den |y| and |y|; the offset's zero components drop out at compile time.
struct LatBond {
    float yx, yy, yz, num, D, ay;
};

template <int OX, int OY, int OZ, int Q>
__device__ __forceinline__ LatBond lat_terms(const StepArgsF32& a, const float3 e)
{
    LatBond r;
    const float tx = OX ? e.x + a.lat_xi2[OX + 3] : e.x;
    const float ty = OY ? e.y + a.lat_xi2[OY + 3] : e.y;
    const float tz = OZ ? e.z + a.lat_xi2[OZ + 3] : e.z;
    r.yx = OX ? e.x + a.lat_xi[OX + 3] : e.x;
    r.yy = OY ? e.y + a.lat_xi[OY + 3] : e.y;
    r.yz = OZ ? e.z + a.lat_xi[OZ + 3] : e.z;
    r.num = fmaf(e.x, tx, fmaf(e.y, ty, e.z * tz));
    const float y2 = r.num + a.lat_q[Q];
    r.ay = y2 * rsqrt_fast(y2);
    r.D = fmaf(r.ay, a.lat_q[Q], a.lat_l[Q] * y2);
    return r;
}

// the same terms for an offset known only at run time (bit for bit the same
// operations: a zero component adds +0, which leaves every sum unchanged)
__device__ __forceinline__ LatBond lat_terms_rt(const StepArgsF32& a, const float3 e, int ox,
                                                int oy, int oz, int q)
{
    LatBond r;
    const float tx = e.x + a.lat_xi2[ox + 3];
    const float ty = e.y + a.lat_xi2[oy + 3];
    const float tz = e.z + a.lat_xi2[oz + 3];
    r.yx = e.x + a.lat_xi[ox + 3];
    r.yy = e.y + a.lat_xi[oy + 3];
    r.yz = e.z + a.lat_xi[oz + 3];
    r.num = fmaf(e.x, tx, fmaf(e.y, ty, e.z * tz));
    const float y2 = r.num + a.lat_q[q];
    r.ay = y2 * rsqrt_fast(y2);
    r.D = fmaf(r.ay, a.lat_q[q], a.lat_l[q] * y2);
    return r;
}

// A bond of slot m whose stretch reached the near-s_c band: decide the break
// (FP32 away from its s_c, the literal FP64 stretch of Eq. 4 near it, then the
// no-fail rule) and return its force term (zero when it breaks).
template <int SCM>
__device__ __noinline__ float3 lat_resolve(const StepArgsF32& a, int cur, int64_t i, int m,
                                           bool* broken)
{
    const int ox = c_stencil.o[m][0], oy = c_stencil.o[m][1], oz = c_stencil.o[m][2];
    const int q = c_stencil.o[m][3];
    const int64_t j = i + (int64_t)ox * a.lat_sx + (int64_t)oy * a.lat_sy + oz;
    const float4* __restrict__ R = a.rec[cur];
    float4 ai, bi, aj, bj;
    ld_rec(R + 2 * i, ai, bi);
    ld_rec(R + 2 * j, aj, bj);
    const LatBond b = lat_terms_rt(a, lat_eta(lat_own(ai, bi), aj, bj), ox, oy, oz, q);
    const double sc = SCM == 1 ? sc_draw(a.sc_seed, a.sc_lo, a.sc_hi, a.gid[i], a.gid[j]) : a.sc;
    const float scf = (float)sc;
    // num |y| - s_c D = den |y| (s - s_c): its sign decides, away from s_c
    const float r = fmaf(-scf, b.D, b.num * b.ay);
    bool brk;
    if (fabsf(r) > a.guard * scf * b.D) {
        brk = r >= 0.0f;
    } else {
        const NodeF32 ni = unpack(ai, bi), nj = unpack(aj, bj);
        const double ui[3] = {(double)ni.hx + (double)ni.lx, (double)ni.hy + (double)ni.ly,
                              (double)ni.hz + (double)ni.lz};
        const double uj[3] = {(double)nj.hx + (double)nj.lx, (double)nj.hy + (double)nj.ly,
                              (double)nj.hz + (double)nj.lz};
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
    if (brk) return make_float3(0.f, 0.f, 0.f);
    const float coef = b.num * rcp_fast(b.D);
    return make_float3(coef * b.yx, coef * b.yy, coef * b.yz);
}

// State of a lane over its node's stencil walk.
struct LatLane {
    LatOwn own;
    const float4* Ri;   // the node's record in the buffer being read
    int64_t i;
    float fx, fy, fz;
    uint32_t word[4];   // bond flags (stencil slot order)
    uint32_t pend;      // near-s_c candidates of the current flag word
    int alive;          // intact bonds after this step's decisions
};

// Slot M: one bond, and after the last slot of a flag word the word's
// near-s_c candidates.
template <int SCM, int M>
__device__ __forceinline__ void lat_slot(const StepArgsF32& a, int cur, LatLane& s)
{
    constexpr Off3 o = stencil_offset(M);
    constexpr int q = M >> 5, b = M & 31;
    if constexpr (b == 0) s.pend = 0u;
    float4 ja, jb;
    ld_rec(s.Ri + 2 * (o.x * a.lat_sx + o.y * a.lat_sy) + 2 * o.z, ja, jb);
    const LatBond t = lat_terms<o.x, o.y, o.z, o.q>(a, lat_eta(s.own, ja, jb));
    const bool alive = (s.word[q] >> b) & 1u;
    const bool cand = t.num >= a.lat_thr[o.q];
    float coef = t.num * rcp_fast(t.D);
    coef = (alive && !cand) ? coef : 0.0f;
    s.pend |= (alive && cand) ? (1u << b) : 0u;
    s.fx = fmaf(coef, t.yx, s.fx);
    s.fy = fmaf(coef, t.yy, s.fy);
    s.fz = fmaf(coef, t.yz, s.fz);
    if constexpr (b == 31 || M == kStencil - 1) {
        uint32_t nword = s.word[q];
        uint32_t pend = s.pend;
        while (pend) {
            const int bb = __ffs(pend) - 1;
            pend &= pend - 1u;
            bool broken;
            const float3 f = lat_resolve<SCM>(a, cur, s.i, 32 * q + bb, &broken);
            if (broken) {
                nword &= ~(1u << bb);
            } else {
                s.fx += f.x;
                s.fy += f.y;
                s.fz += f.z;
            }
        }
        s.word[q] = nword;
        s.alive += __popc(nword);
    }
}

template <int SCM, int... M>
__device__ __forceinline__ void lat_walk(const StepArgsF32& a, int cur, LatLane& s,
                                         std::integer_sequence<int, M...>)
{
    (lat_slot<SCM, M>(a, cur, s), ...);
}

template <int SCM>
__global__ void __launch_bounds__(256, PD_F32_MIN_BLOCKS)
    k_step_f32_lat(const __grid_constant__ StepArgsF32 a)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const int cur = (int)(step & 1);
    const int64_t nslices = (a.n + 31) >> 5;
    const float4* __restrict__ R = a.rec[cur];
    float4* __restrict__ Rout = const_cast<float4*>(a.rec[cur ^ 1]);
    const float wc = a.w_const;

    for (int64_t g = wid; g < nslices; g += nwarps) {
        LatLane s;
        s.i = (g << 5) + lane;
        s.Ri = R + 2 * s.i;
        float4 ai, bi;
        ld_rec(s.Ri, ai, bi);
        const NodeF32 ni = unpack(ai, bi);
        s.own = lat_own(ai, bi);
        uint32_t* bw = a.bits + g * 4 * 32 + lane;
#pragma unroll
        for (int q = 0; q < 4; ++q) s.word[q] = bw[q * 32];
        const uint32_t word0[4] = {s.word[0], s.word[1], s.word[2], s.word[3]};
        s.fx = s.fy = s.fz = 0.f;
        s.pend = 0u;
        s.alive = 0;
        lat_walk<SCM>(a, cur, s, std::make_integer_sequence<int, kStencil>{});
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (s.word[q] != word0[q]) bw[q * 32] = s.word[q];

        // ---- integration of the lane's node (damped Euler-Cromer, Eq. 11),
        // linear displacement ramp, damage (Eq. 8) from the intact-bond count
        const int64_t i = s.i;
        if (i < a.n) {
            const uint32_t cls = a.bcc[i];
            uint32_t mask = 0u;
            const BcClass* bc = nullptr;
            float F[3] = {wc * s.fx, wc * s.fy, wc * s.fz};
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
            st_rec(Rout + 2 * i, make_float4(ni.x, ni.y, ni.z, H[0]),
                   make_float4(H[1], H[2], bf_pack(L[1], L[0]), bf_pack(0.0f, L[2])));
            a.lo32[i] = make_float4(L[0], L[1], L[2], 0.0f);
            const float wi = a.wsum_inv[i];
            const float ws = wc * (float)s.alive;
            a.damage[i] = wi > 0.0f ? fmaxf(0.0f, 1.0f - ws * wi) : 0.0f;
            if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
        }
    }
}

}  // namespace

const void* step_f32_kernel_lat(int sc_mode)
{
    return sc_mode == 0 ? (const void*)k_step_f32_lat<0> : (const void*)k_step_f32_lat<1>;
}

cudaError_t launch_step_f32_lat(const StepArgsF32& a, int sc_mode, int grid, int block,
                                cudaStream_t s)
{
    if (sc_mode == 0)
        k_step_f32_lat<0><<<grid, block, 0, s>>>(a);
    else
        k_step_f32_lat<1><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pd
