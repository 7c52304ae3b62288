// Fused FP32-bulk peridynamic step kernel for sm_103a.
//
// One launch = one explicit time step: bond kinematics (Eq. 4), irreversible
// breaking (Eq. 6), pairwise PMB force (Eq. 5) reduced onto the node
// (Eq. 10), body force, damped Euler-Cromer update (Eq. 11), displacement
// BCs and damage (Eq. 8).  The paper splits this into a bond kernel and an
// integrator kernel because an in-place update would race with neighbours
// still reading u^n (Section 3.3); here the node records that neighbours read
// are double-buffered (step k reads buffer k&1, writes (k+1)&1), so the whole
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
//
// Node record: 32 bytes, one L1/L2 sector, read with one 256-bit load:
//   {x~, y~, z~, h_x | h_y, h_z, bf16(l_x, l_y), bf16(l_z, 0)}
// (lengths in units of the horizon, positions centred).  The displacement is
// an unevaluated float-float sum u/delta = h + l: the owner keeps l in full
// FP32 (private array, exact two-sum updates, 48-bit significand) and
// publishes it rounded to bf16 in the record; eta = (h_j - h_i) + (l_j - l_i)
// is then accurate to ~2^-33 |u/delta|, i.e. to FP32 relative accuracy of eta
// even when |u| is far larger than |eta|.
//
// Precision: bond arithmetic is FP32 with the cancellation-free stretch
// s = eta.(2 xi + eta) / (|xi| (|xi| + |xi+eta|)).  Both directions of a bond
// read the same records and the arithmetic is exactly antisymmetric (j->i sees
// -xi, -eta and produces the same bits), so both break together.  A bond whose
// FP32 stretch is within a relative band of s_c is re-tested with the literal
// FP64 stretch of Eq. 4.
//
// The slot loop is instruction-issue bound (about 60 instructions per bond),
// so the per-bond vector differences run as packed f32x2 operations on the
// register pairs the 256-bit record load delivers: (x, y), (z, h_x),
// (h_y, h_z), (l_x, l_z).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pd_internal.h"

namespace pd {
namespace {

#ifndef PD_F32_UNROLL
#define PD_F32_UNROLL 4
#endif
#ifndef PD_F32_MIN_BLOCKS
#define PD_F32_MIN_BLOCKS 2
#endif
constexpr int kUnroll = PD_F32_UNROLL;  // family slots in flight per lane

// Bilinear-softening build (compiled by pd_step_f32_soft.cu): every slot also
// carries the bond's integrity mu; the fast path scales the force by it, and
// bonds whose stretch reaches the band below s_0 = s_c / kr are resolved like
// the near-s_c ones, where mu is lowered.
#ifndef PD_F32_SOFT
#define PD_F32_SOFT 0
#endif
constexpr bool kSoft = PD_F32_SOFT != 0;

// Extended-epilogue build (pd_step_f32_ext.cu, and the softening build): the
// per-node update also handles velocity-Verlet, the smooth loading start and
// the read-only force pass.  The plain build keeps the Euler-Cromer epilogue
// with the linear loading ramp: the extra branches alone cost the slot loop
// about 9 % in code generation.
#ifndef PD_F32_EXT
#define PD_F32_EXT PD_F32_SOFT
#endif
constexpr bool kExt = PD_F32_EXT != 0;

// State-based build (pd_step_f32_osb.cu): includes this file for its helpers
// and defines the two kernels of the ordinary state-based model there, without
// the bond-based step's public entry points.
#ifndef PD_F32_OSB
#define PD_F32_OSB 0
#endif
// Lattice build (pd_step_f32_lat.cu): the same, for the regular-lattice stencil kernel.
#ifndef PD_F32_LAT
#define PD_F32_LAT 0
#endif

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

// One 32-byte record with a single 256-bit non-coherent load.
__device__ __forceinline__ void ld_rec(const float4* p, float4& a, float4& b)
{
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z),
                   "=f"(b.w)
                 : "l"(p));
}

__device__ __forceinline__ void st_rec(float4* p, const float4& a, const float4& b)
{
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a.x),
                 "f"(a.y), "f"(a.z), "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}

__device__ __forceinline__ float ld_f32(const float* p)
{
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ float bf_lo(float packed)
{
    return __uint_as_float(__float_as_uint(packed) << 16);
}
__device__ __forceinline__ float bf_hi(float packed)
{
    return __uint_as_float(__float_as_uint(packed) & 0xffff0000u);
}
__device__ __forceinline__ float bf_pack(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return __uint_as_float(*reinterpret_cast<const uint32_t*>(&v));
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

// A node as seen by its neighbours: position and published displacement.
struct NodeF32 {
    float x, y, z, hx, hy, hz, lx, ly, lz;
};

__device__ __forceinline__ NodeF32 unpack(const float4 a, const float4 b)
{
    NodeF32 r;
    r.x = a.x;
    r.y = a.y;
    r.z = a.z;
    r.hx = a.w;
    r.hy = b.x;
    r.hz = b.y;
    // b.z = {bf16(l_x) high half, bf16(l_y) low half}: read as a float it is
    // l_x up to a relative 2^-7 of l_x itself (< 2^-31 |h|), so only l_y needs
    // a shift; b.w = {bf16(l_z), 0} is l_z exactly.
    r.lx = b.z;
    r.ly = bf_lo(b.z);
    r.lz = b.w;
    return r;
}

// FP32 bond kinematics in horizon units: y = xi + eta, num = eta.(2 xi + eta)
// = |y|^2 - |xi|^2 (no cancellation), den = |xi| (|xi| + |y|), so s = num / den.
struct BondF32 {
    float yx, yy, yz, num, den, y2;
};

__device__ __forceinline__ BondF32 bond_f32(const NodeF32& i, const NodeF32& j)
{
    BondF32 r;
    const float ex = j.x - i.x, ey = j.y - i.y, ez = j.z - i.z;
    const float hx = (j.hx - i.hx) + (j.lx - i.lx);
    const float hy = (j.hy - i.hy) + (j.ly - i.ly);
    const float hz = (j.hz - i.hz) + (j.lz - i.lz);
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

// The lane's own record, negated and paired as the 256-bit load delivers
// registers: (x, y), (z, h_x), (h_y, h_z), (l_x, l_z), plus l_y.
struct LanePairs {
    float2 xy, zhx, hyz, lxz;
    float ly;
};

__device__ __forceinline__ LanePairs lane_pairs(const float4 a, const float4 b)
{
    LanePairs p;
    p.xy = make_float2(-a.x, -a.y);
    p.zhx = make_float2(-a.z, -a.w);
    p.hyz = make_float2(-b.x, -b.y);
    p.lxz = make_float2(-b.z, -b.w);
    p.ly = -bf_lo(b.z);
    return p;
}

// bond_f32 with the vector differences done as packed f32x2 operations on the
// record's register pairs (the same IEEE operations in the same order per
// component, so j->i still mirrors i->j bit for bit)
__device__ __forceinline__ BondF32 bond_f32_pk(const LanePairs& i, const float4 ja, const float4 jb)
{
    BondF32 r;
    const float2 exy = __fadd2_rn(make_float2(ja.x, ja.y), i.xy);
    const float2 ezhx = __fadd2_rn(make_float2(ja.z, ja.w), i.zhx);
    const float2 dhyz = __fadd2_rn(make_float2(jb.x, jb.y), i.hyz);
    const float2 dlxz = __fadd2_rn(make_float2(jb.z, jb.w), i.lxz);
    const float dly = bf_lo(jb.z) + i.ly;
    const float2 hxy = make_float2(ezhx.y + dlxz.x, dhyz.x + dly);
    const float hz = dhyz.y + dlxz.y;
    const float ez = ezhx.x;
    const float2 yxy = __fadd2_rn(exy, hxy);
    const float yz = ez + hz;
    const float2 sxy = __fadd2_rn(exy, yxy);
    const float2 e2 = __fmul2_rn(exy, exy);
    const float xx = fmaf(ez, ez, e2.x + e2.y);
    const float2 n2 = __fmul2_rn(hxy, sxy);
    r.num = fmaf(hz, ez + yz, n2.x + n2.y);
    r.yx = yxy.x;
    r.yy = yxy.y;
    r.yz = yz;
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

// weight c V of node j; with uniform weights (per instance in a batch: both ends
// of a bond belong to the same instance) it is the lane's constant wc
template <bool UW>
__device__ __forceinline__ float node_w(const StepArgsF32& a, int64_t j, float wc)
{
    return UW ? wc : __ldg(a.w + j);
}

__device__ __forceinline__ float lane_wconst(const StepArgsF32& a, int64_t i)
{
    return a.inst != nullptr ? a.itab[a.inst[i]].w_const : a.w_const;
}

// A bond whose FP32 stretch reached the band just below the smallest s_c: the
// break test is decided in FP32 when s is clearly away from the bond's s_c and
// otherwise with the literal FP64 stretch of Eq. 4 (FP64 positions, published
// float-float displacement, read identically by both directions); the no-fail
// rule applies last.  Returns the bond's force contribution {fx, fy, fz, w},
// all zero when it breaks (*broken = true).
template <int SCM, bool UW>
__device__ __noinline__ float4 resolve_bond(const StepArgsF32& a, int cur, int64_t i, int64_t j,
                                            int64_t slot, bool* broken)
{
    const float4* __restrict__ R = a.rec[cur];
    float4 ai, bi, aj, bj;
    ld_rec(R + 2 * i, ai, bi);
    ld_rec(R + 2 * j, aj, bj);
    const NodeF32 ni = unpack(ai, bi), nj = unpack(aj, bj);
    const BondF32 b = bond_f32(ni, nj);
    double sc = a.sc;
    if (a.inst != nullptr) {  // batch: the instance's own parameters, local ids as keys
        const InstParams& ip = a.itab[a.inst[i]];
        sc = ip.sc_mode == 1 ? sc_draw(ip.sc_seed, ip.sc_lo, ip.sc_hi, a.hid[i], a.hid[j]) : ip.sc;
    } else if (SCM == 1) {
        sc = sc_draw(a.sc_seed, a.sc_lo, a.sc_hi, a.gid[i], a.gid[j]);
    }
    const float scf = (float)sc;
    const float r = fmaf(-scf, b.den, b.num);  // den * (s - s_c)
    bool brk;
    if (fabsf(r) > a.guard * scf * b.den) {
        brk = r >= 0.0f;
    } else {
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
    if (brk) {
        if (kSoft) a.integ[slot] = 0.0f;
        return make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float wv = node_w<UW>(a, j, UW ? lane_wconst(a, i) : 0.0f);
    float w = wv;
    if (a.cbond != nullptr) w *= a.cbond[slot];
    float mu = 1.0f;
    if (kSoft) {
        // integrity only decreases, as the stretch passes s_0 (0 for a no-fail
        // bond past s_c); the fast path applies the stored value
        mu = a.integ[slot];
        const double s = (double)(b.num / b.den), s0 = sc / a.kr;
        if (s > s0) {
            const float ms = s >= sc ? 0.0f : (float)soft_mu_of(s, s0, sc, a.k1, a.beta);
            if (ms < mu) {
                mu = ms;
                a.integ[slot] = ms;
            }
        }
        w *= mu;
    }
    const float coef = bond_coef(b, w);
    // .w: the damage weight (w V; for uniform weights the integrity alone)
    return make_float4(coef * b.yx, coef * b.yy, coef * b.yz, kSoft ? (UW ? mu : wv * mu) : wv);
}

template <int SCM, bool UW>
__global__ void __launch_bounds__(256, PD_F32_MIN_BLOCKS)
    k_step_f32(const __grid_constant__ StepArgsF32 a)
{
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t step = a.step_ctr[0] + a.k;
    const int cur = (int)(step & 1);
    const int Q = a.Q;
    const int64_t W = 32LL * Q;
    const int64_t nslices = (a.n + 31) >> 5;
    const float4* __restrict__ R = a.rec[cur];
    float4* __restrict__ Rout = const_cast<float4*>(a.rec[cur ^ 1]);
    const float* __restrict__ cb = a.cbond;

    for (int64_t g = wid; g < nslices; g += nwarps) {
        const int Wg = a.sw[g];
        const int32_t* __restrict__ col = a.nbr + g * W * 32 + lane;
        if (lane == 0) prefetch_l2(col, (uint32_t)(((Wg + 3) & ~3) * 128));
        const int64_t i = (g << 5) + lane;
        // band just below the smallest s_c the node's bonds can have (per
        // instance in a batch; both ends of a bond belong to the same instance)
        const float fast_lo = a.inst != nullptr ? a.itab[a.inst[i]].fast_lo : a.fast_lo;
        const float wc = UW ? lane_wconst(a, i) : 0.0f;
        float4 ai, bi;
        ld_rec(R + 2 * i, ai, bi);
        const NodeF32 ni = unpack(ai, bi);
        const LanePairs pi = lane_pairs(ai, bi);
        uint32_t* bw = a.bits + g * Q * 32 + lane;
        float fx = 0.f, fy = 0.f, fz = 0.f, ws = 0.f;
        int alive_count = 0;

        // Slots are visited in chunks of kUnroll; the neighbour ids of the next
        // chunk are loaded while the current chunk's records are gathered and
        // evaluated, so the id stream's latency overlaps the arithmetic.  Every
        // slot is evaluated; slots of broken bonds or beyond a lane's family (id =
        // the node itself) are masked with selects, so the warp never diverges.
        const int nch = (Wg + kUnroll - 1) / kUnroll;
        int32_t jn[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) jn[u] = __ldg(col + u * 32);
        uint32_t word = 0u, nword = 0u, pend = 0u;
        for (int c = 0; c < nch; ++c) {
            const int m0 = c * kUnroll;
            const int q = m0 >> 5, b0 = m0 & 31;
            if (b0 == 0) {
                word = bw[q * 32];
                nword = word;
                pend = 0u;  // members in the near-s_c band, resolved at the word's end
            }
            int32_t jj[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) jj[u] = jn[u];
            if (c + 1 < nch) {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) jn[u] = __ldg(col + (m0 + kUnroll + u) * 32);
            }
            float4 ra[kUnroll], rb[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) ld_rec(R + 2 * (int64_t)jj[u], ra[u], rb[u]);
            const uint32_t wb = word >> b0;
            uint32_t pc = 0u;
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const bool alive = (wb >> u) & 1u;
                const BondF32 bd = bond_f32_pk(pi, ra[u], rb[u]);
                // near-s_c candidates; unused/broken slots are dropped from the
                // pending set once per chunk (pc & wb below)
                const bool cand = bd.num >= fast_lo * bd.den;
                pc |= cand ? (1u << u) : 0u;
                float wj = node_w<UW>(a, jj[u], wc);
                const float wv = wj;
                if (cb != nullptr) wj *= ld_f32(cb + (g * W + m0 + u) * 32 + lane);
                float mj = 1.0f;
                if (kSoft) {
                    mj = ld_f32(a.integ + (g * W + m0 + u) * 32 + lane);
                    wj *= mj;
                }
                float coef = bond_coef(bd, wj);
                coef = cand ? 0.0f : coef;
                coef = alive ? coef : 0.0f;
                fx = fmaf(coef, bd.yx, fx);
                fy = fmaf(coef, bd.yy, fy);
                fz = fmaf(coef, bd.yz, fz);
                if (kSoft)
                    ws += (alive && !cand) ? (UW ? mj : wv * mj) : 0.0f;
                else if (!UW)
                    ws += (alive && !cand) ? wv : 0.0f;
            }
            pend |= (pc & wb) << b0;
            if (b0 + kUnroll == 32 || c + 1 == nch) {  // end of bond-flag word q
                while (pend) {
                    const int b = __ffs(pend) - 1;
                    pend &= pend - 1u;
                    const int64_t slot = (g * W + q * 32 + b) * 32 + lane;
                    bool broken;
                    const float4 f = resolve_bond<SCM, UW>(a, cur, i, col[(int64_t)(q * 32 + b) * 32],
                                                           slot, &broken);
                    if (broken) {
                        nword &= ~(1u << b);
                    } else {
                        fx += f.x;
                        fy += f.y;
                        fz += f.z;
                        if (kSoft || !UW) ws += f.w;
                    }
                }
                if (nword != word) bw[q * 32] = nword;
                alive_count += __popc(nword);
            }
        }
        if (UW) ws = kSoft ? wc * ws : wc * (float)alive_count;

        // ---- integration of the lane's node (damped Euler-Cromer, Eq. 11, or
        // damped velocity-Verlet)
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
            // velocity-Verlet: a^n is formed afresh at the step the state was set
            const bool first = kExt && a.vv && step == a.step_ctr[1];
            const float dtd = (float)(a.dt * a.inv_delta);
            const float4 lo = a.lo32[i];
            float H[3] = {ni.hx, ni.hy, ni.hz};
            float L[3] = {lo.x, lo.y, lo.z};
            bool finite = true;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // stored velocity: v^n (Euler-Cromer) or, for velocity-Verlet, the
                // half-step velocity v^{n-1} + dt/2 a^{n-1} (v^n right after a set state)
                const float vi = a.v[3 * i + c];
                if constexpr (!kExt) {
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
                } else {
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
            }
            if (kExt && a.peek) continue;
            st_rec(Rout + 2 * i, make_float4(ni.x, ni.y, ni.z, H[0]),
                   make_float4(H[1], H[2], bf_pack(L[1], L[0]), bf_pack(0.0f, L[2])));
            a.lo32[i] = make_float4(L[0], L[1], L[2], 0.0f);
            const float wi = a.wsum_inv[i];
            // clamp: ws * (1 / sum w) can round to 1 + 1 ulp for an intact family
            a.damage[i] = wi > 0.0f ? fmaxf(0.0f, 1.0f - ws * wi) : 0.0f;
            if (!finite) atomicOr(a.err, PD_DEVERR_NONFINITE);
        }
    }
}

template <int SCM, bool UW>
cudaError_t launch_v(const StepArgsF32& a, int grid, int block, cudaStream_t s)
{
    k_step_f32<SCM, UW><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

#if !PD_F32_OSB && !PD_F32_LAT
#if PD_F32_SOFT
#define PD_F32_KERNEL_OF step_f32_kernel_soft
#define PD_F32_LAUNCH launch_step_f32_soft
#elif PD_F32_EXT
#define PD_F32_KERNEL_OF step_f32_kernel_ext
#define PD_F32_LAUNCH launch_step_f32_ext
#else
#define PD_F32_KERNEL_OF step_f32_kernel
#define PD_F32_LAUNCH launch_step_f32
#endif

// per_bond_c selects no separate variant (it is a uniform run-time branch)
const void* PD_F32_KERNEL_OF(int sc_mode, bool uniform_w, bool /*per_bond_c*/)
{
    if (sc_mode == 0)
        return uniform_w ? (const void*)k_step_f32<0, true> : (const void*)k_step_f32<0, false>;
    return uniform_w ? (const void*)k_step_f32<1, true> : (const void*)k_step_f32<1, false>;
}

cudaError_t PD_F32_LAUNCH(const StepArgsF32& a, int sc_mode, int grid, int block, cudaStream_t s)
{
    if (sc_mode == 0)
        return a.uniform_w ? launch_v<0, true>(a, grid, block, s) : launch_v<0, false>(a, grid, block, s);
    return a.uniform_w ? launch_v<1, true>(a, grid, block, s) : launch_v<1, false>(a, grid, block, s);
}
#endif  // !PD_F32_OSB && !PD_F32_LAT

}  // namespace pd
