// Internal declarations of the peridynamic step library (not installed).
//
// Device layout.  Nodes are in the library's node order p = 0..n-1 (the
// caller's order, or a cell-sorted order on request), padded to n_pad, a
// multiple of 32.  Slice g = nodes 32g..32g+31; warp lane l of a slice owns
// node p = 32g + l.
//   nbr   int32 sliced ELL ("SELL-32"): member m of node p at
//         nbr[(g*W + m)*32 + l], W = 32*Q slots per node; members ascending by
//         node index; unused slots hold p.  A warp reads slot m of its 32 nodes
//         with one coalesced 128-byte load.
//   bits  uint32 bond flags: word q of node p at bits[(g*Q + q)*32 + l]; bit b of
//         word q is member 32q+b (1 = intact).  Unused slots are 0.
//   sw    int32 per slice: largest family size in the slice (loop bound).
//   bcc   uint8 boundary-condition class per node -> BcClass table
//   gid   int32 caller id of each node (padding: 0)
//   x64   FP64 reference coordinates (3 per node)
//   wsum_inv  1 / sum_j w_j over the family after the initial cuts
//   damage    per node, rewritten by every step
//   step_ctr  int64 device step counter (read by every step kernel)
//   err       int32 device error bits (PD_DEVERR_*)
// FP32-bulk path (all lengths in units of the horizon, positions centred):
//   rec[2] 32-byte node records (one sector), double buffered:
//          {x~, y~, z~, hx | hy, hz, bf16(lx, ly), bf16(lz, 0)}: reference position
//          and the displacement u~ = h + l as published to neighbours
//   lo32   float4 {lx, ly, lz, 0}: the owner's full-precision l (the float-float
//          pair h + l has a 48-bit significand and is the integrator's state)
//   w      float per node: c V (constant c) or V (per-bond c)
//   v      float velocity, 3 per node, updated in place by its owner
// FP64 path:
//   rec[2] 8 doubles per node {x, y, z, w, ux, uy, uz, 0}, double buffered
//   v      double velocity, 3 per node
//   (PD_PREC_DW handles add 64-byte double-word copies of the records for the
//   neighbours and a double-word reference length per slot, see DwArgs)
#pragma once

#include <cstdint>
#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>

#define PD_DEVERR_NONFINITE 1
#define PD_DEVERR_TIMEOUT 2  // a bounded device wait ran out

namespace pd {

struct BcClass {
    uint32_t mask;     // bit a (0..2): component a displacement-controlled; bit 3: no-fail
    uint32_t pad;
    double disp[3];    // prescribed displacement per unit scale
    double force[3];   // body-force density per unit load
};

// Critical-stretch parameters of one instance of a batch.
struct InstParams {
    int32_t sc_mode;           // 0 constant, 1 per-bond draw
    float fast_lo;             // (1 - 2 guard) * sc_lo (FP32 kernel fast path)
    float w_const;             // c V of the instance when its volumes are uniform
    float pad;
    double sc, sc_lo, sc_hi;
    uint64_t sc_seed;
    // a batch of regular-lattice models (the stencil kernel): each instance's
    // state in units of its own spacing dx, its node-order strides
    int32_t lat_sx, lat_sy;
    float lat_thr_t;           // fast_lo (2 + fast_lo): s >= fast_lo <=> num >= q lat_thr_t
    float lat_cc_t, lat_ch_t;  // the stencil walk's candidate test |num - q cc_t| >= q ch_t
                               // (lat_cc, lat_ch of StepArgsF32 per unit q)
    float dtd;                 // dt / dx
    double unit, inv_unit;     // dx, 1 / dx
};

// Regular-lattice stencil.  On a cubic lattice of spacing dx with
// 3 dx <= delta < sqrt(10) dx, the family of Eq. 9 of an interior node is the
// set of the 122 integer offsets o with 0 < |o|^2 <= 9 (in units of dx); a
// node near a face or a cut has a subset of them.  A lattice model's layout
// gives each offset a fixed slot (of 128: 4 flag words of 32 bits).  The
// offsets are grouped in "rows" (o_x, o_y fixed, o_z running), rows of equal
// q_xy = o_x^2 + o_y^2 in segments, and the segments laid out so that no row
// crosses a flag word:
//   word 0: q_xy = 1 (4 rows, o_z = -2..2), q_xy = 8 (4 rows, o_z = -1..1)
//   word 1: q_xy = 2 (4 rows, -2..2), q_xy = 0 (o_z = +-1..3), q_xy = 9 (4 rows, o_z = 0)
//   word 2: q_xy = 4 (4 rows, -2..2), q_xy = 5 (rows 0-1, -2..2)
//   word 3: q_xy = 5 (rows 2-7, -2..2)
// Within a q_xy the rows with o_y = 0 come first, then those with o_x = 0, then
// the rest, each group in lexicographic (o_x, o_y) order; a segment holds rows
// of one such group, so that its zero components are known.  Slots 62, 63, 94,
// 95, 126 and 127 are unused.  The stencil kernel walks a segment of 5-offset
// rows as a loop over its rows with the o_z offsets unrolled, and the short
// rows (q_xy = 0, 8, 9) unrolled.
constexpr int kStencil = 122;
// |x| = |num| / |xi|^2 up to which the stencil walk's series coefficient is used
// (truncation error below 0.25 ulp of FP32); bonds past it are corrected exactly
constexpr double kLatPolyX = 3e-3;
constexpr int kStencilSlots = 128;
constexpr int kStencilR2 = 9;
constexpr int kStencilSegs = 10;
constexpr int kStencilRows = 29;
struct Off3 {
    int x, y, z, q;  // q = |o|^2; q = 0 marks an unused slot
};
struct StencilSeg {
    int qxy;      // o_x^2 + o_y^2 of its rows
    int row0;     // first row (of the rows with this q_xy, in the order above)
    int nrows;
    int word;     // flag word
    int bit0;     // first bit in the word
    int first;    // index of its first row among all kStencilRows rows
    int zx, zy;   // 1: o_x (o_y) is 0 in every row of the segment
    int unroll;   // 1: rows unrolled in the kernel, 0: a loop over the rows
};
__host__ __device__ constexpr int stencil_row_len(int qxy)
{
    return qxy == 0 ? 6 : qxy == 8 ? 3 : qxy == 9 ? 1 : 5;
}
// o_z of position k in a row
__host__ __device__ constexpr int stencil_row_oz(int qxy, int k)
{
    return qxy == 0 ? (k < 3 ? k - 3 : k - 2) : k - (stencil_row_len(qxy) - 1) / 2;
}
// (o_x, o_y) of row r among the rows with o_x^2 + o_y^2 = qxy: o_y = 0 first,
// then o_x = 0, then the others, each lexicographic
__host__ __device__ constexpr Off3 stencil_row_xy(int qxy, int r)
{
    int k = 0;
    for (int grp = 0; grp < 3; ++grp)
        for (int a = -3; a <= 3; ++a)
            for (int b = -3; b <= 3; ++b) {
                if (a * a + b * b != qxy) continue;
                const int g = b == 0 ? 0 : a == 0 ? 1 : 2;
                if (g != grp) continue;
                if (k == r) return Off3{a, b, 0, qxy};
                ++k;
            }
    return Off3{0, 0, 0, 0};
}
__host__ __device__ constexpr StencilSeg stencil_seg(int sg)
{
    constexpr int q[kStencilSegs] = {1, 1, 8, 2, 0, 9, 4, 4, 5, 5};
    constexpr int r0[kStencilSegs] = {0, 2, 0, 0, 0, 0, 0, 2, 0, 2};
    constexpr int nr[kStencilSegs] = {2, 2, 4, 4, 1, 4, 2, 2, 2, 6};
    constexpr int w[kStencilSegs] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3};
    constexpr int b[kStencilSegs] = {0, 10, 20, 0, 20, 26, 0, 10, 20, 0};
    constexpr int zx[kStencilSegs] = {0, 1, 0, 0, 1, 0, 0, 1, 0, 0};
    constexpr int zy[kStencilSegs] = {1, 0, 0, 0, 1, 0, 1, 0, 0, 0};
    constexpr int un[kStencilSegs] = {0, 0, 1, 0, 1, 1, 0, 0, 0, 0};
    int first = 0;
    for (int k = 0; k < sg; ++k) first += nr[k];
    return StencilSeg{q[sg], r0[sg], nr[sg], w[sg], b[sg], first, zx[sg], zy[sg], un[sg]};
}
// the offset of slot m (q = 0: unused slot)
__host__ __device__ constexpr Off3 stencil_offset(int m)
{
    for (int sg = 0; sg < kStencilSegs; ++sg) {
        const StencilSeg s = stencil_seg(sg);
        const int len = stencil_row_len(s.qxy);
        const int start = 32 * s.word + s.bit0;
        if (m >= start && m < start + len * s.nrows) {
            const int r = (m - start) / len, k = (m - start) % len;
            const Off3 xy = stencil_row_xy(s.qxy, s.row0 + r);
            const int oz = stencil_row_oz(s.qxy, k);
            return Off3{xy.x, xy.y, oz, s.qxy + oz * oz};
        }
    }
    return Off3{0, 0, 0, 0};
}
// (o_x, o_y) of row j of all kStencilRows rows, in segment order
__host__ __device__ constexpr Off3 stencil_row(int j)
{
    for (int sg = 0; sg < kStencilSegs; ++sg) {
        const StencilSeg s = stencil_seg(sg);
        if (j >= s.first && j < s.first + s.nrows) return stencil_row_xy(s.qxy, s.row0 + j - s.first);
    }
    return Off3{0, 0, 0, 0};
}

struct StepArgsF32 {
    const int32_t* inst;       // batch: instance of each node, or nullptr
    const InstParams* itab;    // batch: per-instance s_c parameters
    const int32_t* hid;        // batch: instance-local node id (key of the s_c draw)
    const float4* rec[2];      // 2 float4 (32 B) per node
    float4* lo32;              // owner-private full-precision l, 1 float4 per node
    const float* w;            // per-node weight w = c V (or V with per-bond c)
    float w_const;             // the common weight when uniform_w
    int32_t uniform_w;         // all w equal: w_const is used, damage by bit counts
    float* v;
    const int32_t* nbr;
    uint32_t* bits;
    const int32_t* sw;
    const float* cbond;        // SELL layout like nbr, or nullptr
    const uint8_t* bcc;
    const BcClass* bct;
    const int32_t* gid;
    const double* x64;
    const float* wsum_inv;
    float* damage;
    int* err;
    const int64_t* step_ctr;
    int64_t n;
    int32_t k;                 // offset of this launch from the device step counter
    int64_t step_abs;          // lattice kernels: >= 0, the absolute step of a direct
                               // launch, which then sets the counter to step_abs + 1
                               // instead of reading it; -1: counter + k
    int32_t Q;
    int32_t has_nofail;
    int32_t pad0;
    float sc_f;                // constant s_c
    float sc_lo_f;             // lower bound of s_c (= s_c when constant)
    float fast_lo;             // (1 - guard) * sc_lo: below this nothing can break
    float guard;               // relative band around s_c re-tested in FP64
    double sc, sc_lo, sc_hi;
    uint64_t sc_seed;
    double dt, eta, rho, disp_rate, load, delta, inv_delta;
    int64_t ramp_steps;        // smooth loading start over this many steps (0 = linear)
    int32_t vv;                // 1: damped velocity-Verlet, 0: damped Euler-Cromer
    int32_t peek;              // 1: forces and full-step velocity into vout only
    float* vout;               // peek: 3 floats per node (library order)
    float* integ;              // bilinear softening: per-slot integrity mu, or nullptr
    double kr;                 // s_0 = s_c / kr
    double k1, beta;           // trilinear: kink at s_1 = k1 s_0 with force beta c s_0 (k1 > 1)
    // regular-lattice stencil kernel (pd_step_f32_lat.cu); node p = (ix Ny + iy) Nz + iz
    int32_t lat_sx, lat_sy;    // node-order strides of x and y (z: 1)
    float4 lat_rxi[kStencilRows];   // per row (segment order): kappa (o_x, o_y, 2 o_x, 2 o_y)
    int32_t lat_roff[kStencilRows]; // per row: node offset o_x Sx + o_y Sy
    int32_t lat_rox[kStencilRows], lat_roy[kStencilRows];  // per row: o_x, o_y (batches)
    float lat_xi[7];           // kappa c for c = -3..3 (kappa = dx / delta: xi in horizon units)
    float lat_xi2[7];          // 2 kappa c
    float lat_q[kStencilR2 + 1];    // |xi|^2 = kappa^2 q for q = |o|^2
    float lat_l[kStencilR2 + 1];    // |xi| = kappa sqrt(q)
    float lat_thr[kStencilR2 + 1];  // num threshold of the near-s_c band: s >= fast_lo
                                    // <=> num >= fast_lo (2 + fast_lo) |xi|^2
    // the walk's force coefficient num / D as num (pc0 + pc1 num + pc2 num^2), the
    // series of num / D in x = num / |xi|^2 to x^2 (kLatPolyX: its range); the
    // candidates: |num - cc| >= ch, i.e. num >= min(thr, pt) or num <= -pt, with
    // pt = kLatPolyX |xi|^2 (the near-s_c band and the bonds past the series)
    float lat_pc[3][kStencilR2 + 1];
    // the state-based dilation loop's |xi| e~ = |xi| (|y| - |xi|) as num (dc0 + dc1 num
    // + dc2 num^2), its series in x to x^2 (dc0 = 1/2, dc1 = -1 / (8 |xi|^2),
    // dc2 = 1 / (16 |xi|^4)), the same candidates
    float lat_dc[3][kStencilR2 + 1];
    float lat_cc[kStencilR2 + 1], lat_ch[kStencilR2 + 1], lat_pt[kStencilR2 + 1];
    // the bond-based walk takes its bonds two at a time (paired FP32 instructions):
    // per first row j of a row pair, kappa (o_x(j), o_x(j+1), o_y(j), o_y(j+1)) and
    // twice that; per q, pc0, pc1, pc2 and -cc, each twice (one register pair)
    float4 lat_rxp[kStencilRows][2];
    float2 lat_pcd[3][kStencilR2 + 1];
    float2 lat_ccd[kStencilR2 + 1];
    float2 lat_dcd[3][kStencilR2 + 1];  // the state-based dilation loop's dc0..dc2
    // the state-based force loop's |xi| / |y| = 1 + fa0 num + fa1 num^2 and
    // e~ / |y| = num (fb0 + fb1 num + fb2 num^2), the series of (1 + x)^(-1/2) and of
    // 1 - (1 + x)^(-1/2) in x = num / |xi|^2 to x^2 (within 0.25 ulp for |x| <= kLatPolyX),
    // each coefficient twice (one register pair)
    float2 lat_fad[2][kStencilR2 + 1], lat_fbd[3][kStencilR2 + 1];
    float dt_f, eta_f, rho_f;  // dt, eta, rho rounded to FP32 once, on the host
    float dtd_f;               // dt / delta (velocity to displacement in horizon units)
    // regular-lattice models keep their state differently (no rec / lo32):
    double* lat_u[2];          // u / delta in FP64, 3 per node, double buffered
    const float4* lat_pub[2];  // {u_x, u_y, u_z} / delta rounded to FP32, what the
                               // neighbours read (16 B per node, zero halo), double buffered
};

struct StepArgsF64 {
    const int32_t* inst;       // batch: instance of each node, or nullptr
    const InstParams* itab;
    const int32_t* hid;
    const double* rec[2];      // 8 doubles per node
    double* v;
    const int32_t* nbr;
    uint32_t* bits;
    const int32_t* sw;
    int32_t frozen;            // 1: no bond breaks (the adjoint's forward runs)
    int32_t pad1;
    const double* cbond;
    const double* ilen;        // per slot 1 / |xi| (reference bond length)
    const uint8_t* bcc;
    const BcClass* bct;
    const int32_t* gid;
    const double* wsum_inv;
    double* damage;
    int* err;
    const int64_t* step_ctr;
    int64_t n;
    int32_t k;
    int32_t Q;
    int32_t has_nofail;
    int32_t pad0;
    double sc, sc_lo, sc_hi;
    uint64_t sc_seed;
    double dt, eta, rho, disp_rate, load;
    int64_t ramp_steps;        // smooth loading start over this many steps (0 = linear)
    int32_t vv;                // 1: damped velocity-Verlet, 0: damped Euler-Cromer
    int32_t peek;              // 1: forces and full-step velocity into vout only
    double* vout;              // peek: 3 doubles per node (library order)
    double* integ;             // bilinear softening: per-slot integrity mu, or nullptr
    double kr;                 // s_0 = s_c / kr
    double k1, beta;           // trilinear: kink at s_1 = k1 s_0 with force beta c s_0 (k1 > 1)
};

// Double-word (FP64-grade) step of FP64 handles created with PD_PREC_DW
// (pd_step_dw.cu): neighbour records and per-slot reference lengths
struct DwArgs {
    const float4* rec[2];      // 4 float4 per node, double buffered like the FP64 records
    const float2* len;         // per slot |xi| / delta as a double-word (hi, lo)
    const float2* cb;          // per slot stiffness c_ij as a double-word, or nullptr
    double inv_delta;          // 1 / delta
    double w_const;            // c V when the node weights are uniform
    double dt_rho;             // dt / rho
    float fast_lo;             // leading stretch words below this are decided without s_c
                               // (+inf while the bond flags are frozen)
    int32_t uniform_w;         // 1: every node has weight w_const
};

// Ordinary state-based (linear solid) arrays, FP64 handles with model 1
struct OsbArgs {
    double* len;               // per slot |xi|
    const double* vol;         // per node V
    double* mvol;              // per node weighted volume m_i
    double* theta;             // per node dilation of the current step
    double* alpha;             // per node 3 K theta / m - beta theta / 3 (current step)
    double* beta;              // per node 15 G / m
    double K, G;               // bulk and shear modulus
};

// Ordinary state-based arrays of PD_PREC_DW handles (pd_step_osb_dw.cu; lengths
// in horizon units)
struct OsbDwArgs {
    const float2* len;         // per slot |xi| / delta (the double-word step's)
    const double* vol;         // per node V
    double* mvol;              // per node m~ = sum |xi~|^2 V_j
    double* theta;             // per node dilation of the current step
    float4* ab;                // per node {alpha~ h, l, beta~ h, l} (double-words)
    double K, G;
};

cudaError_t launch_osb_dw_setup(const StepArgsF64& a, const OsbDwArgs& o, cudaStream_t s);
cudaError_t launch_osb_dw_step(const StepArgsF64& a, const DwArgs& d, const OsbDwArgs& o, int grid,
                               int block, cudaStream_t s);

// Shared-memory tile step of single bond-based lattice models
// (pd_step_f32_lat_tma.cu): a block per box of BZ x BY x BX nodes, the box's
// records and a halo of 3 nodes copied by one tiled bulk tensor copy.  The
// compiled box shapes (BZ, BY, BX): 0 = (16, 2, 8), 1 = (8, 4, 8), 2 = (32, 2, 4).
constexpr int kLatTmaShapes = 3;
__host__ __device__ constexpr int lat_tma_dim(int shape, int axis)
{
    constexpr int d[kLatTmaShapes][3] = {{16, 2, 8}, {8, 4, 8}, {32, 2, 4}};
    return d[shape][axis];
}
__host__ __device__ constexpr uint32_t lat_tma_tile_bytes(int bz, int by, int bx)
{
    return 16u * (uint32_t)((bz + 6) * (by + 6) * (bx + 6));
}
// dynamic shared memory of a block: the tile, 128 bytes to align it, the barrier
__host__ __device__ constexpr size_t lat_tma_smem_bytes(int shape)
{
    return lat_tma_tile_bytes(lat_tma_dim(shape, 0), lat_tma_dim(shape, 1), lat_tma_dim(shape, 2)) +
           128 + 16;
}
struct LatTmaArgs {
    CUtensorMap map[2];   // the published records of buffer 0 / 1 as the 4-D tensor
                          // {4 floats, Nz, Ny, Nx}, box {4, BZ + 6, BY + 6, BX + 6}
    int32_t nz, ny, nx;   // lattice dimensions
    int32_t tiles_z, tiles_y, tiles_x;
    int32_t extra_tx;     // bytes the barrier waits for beyond the copy's (0; a test
                          // sets it to run the bounded wait out)
};
const void* step_f32_kernel_lat_tma(int shape, int sc_mode, bool per_bond_c);
cudaError_t launch_step_f32_lat_tma(const StepArgsF32& a, const LatTmaArgs& t, int shape,
                                    int sc_mode, int grid, cudaStream_t s);

// Ordinary state-based arrays of FP32 lattice models (pd_step_f32_lat_osb.cu)
struct OsbLatArgs {
    const float4* coef;  // per node {3 / m~, (3K - 5G) / (delta m~), 15 G / (delta m~), 0}
    float4* rec;         // per node the force loop's record {h, A} (zero halo)
    const float* bco;    // per node B = 15 G / (delta m~) (zero halo)
    float* theta;        // per node dilation of the current step
    uint8_t* exact;      // per slice of 32 nodes: 1 when a node of it has a dilation
                         // candidate (the force loop then forms 1 / |y| and e~ exactly)
};
cudaError_t launch_osb_lat_step(const StepArgsF32& a, const OsbLatArgs& o, int sc_mode, int grid,
                                int grid_force, int block, cudaStream_t s);
const void* osb_lat_force_kernel();
const void* osb_lat_dilation_kernel(int sc_mode);

// Ordinary state-based arrays of FP32 handles (lengths in horizon units;
// alpha, beta multiplied by delta, see pd_step_f32.cu)
struct OsbArgs32 {
    float* mvol;   // weighted volume m (horizon units)
    float* theta;  // dilation
    float2* ab;    // (alpha', beta') per node: one 8-byte gather per neighbour
    double K, G, delta;
};

// Arguments of one reverse step of the FP64 adjoint (pd_adjoint.cu); node arrays
// in library order, n_pad entries.
struct AdjArgs {
    const double* x64;         // reference positions (3 per node)
    const double* un;          // u^n, the state the forward step n -> n+1 read
    const double* w;           // vbar + dt ubar (controlled components zeroed)
    const double* ubm;         // ubar of step n+1, controlled components zeroed
    double* ub_out;            // ubar^n
    double* vb_out;            // vbar^n
    const int32_t* nbr;
    const uint32_t* bits;      // frozen bond flags
    const int32_t* sw;
    int32_t Q;
    int32_t pad0;
    const double* vol;         // volumes V
    const double* cbond;       // per-slot stiffness, or nullptr for the constant c
    const double* ilen;        // per slot 1 / |xi|
    double c;
    double* gc;                // per-slot dL/dc accumulator
    double* gl;                // per-node accumulator of force . w
    const uint8_t* bcc;
    const BcClass* bct;
    double dt_rho;             // dt / rho
    double damp;               // 1 - dt eta / rho
    int64_t n;
};

// Reverse step of PD_PREC_DW handles (pd_adjoint_dw.cu): double-word records
// of u^n and w for the neighbours, FP64 node outputs
struct AdjDwArgs {
    const float4* rec;         // 4 float4 per node: positions, u^n / delta, V
    const float4* wrec;        // 2 float4 per node: w
    const float2* len;         // per slot |xi| / delta
    const float2* cb;          // per slot c_ij, or nullptr for the constant c
    float2 c;                  // the constant c as a double-word
    float2* gc;                // per slot dL/dc accumulator, without dt/rho
    const double* w;           // w (FP64)
    const double* ubm;         // ubar of step n+1, controlled components zeroed
    double* ub_out;            // ubar^n
    double* vb_out;            // vbar^n
    double* gl;                // per-node accumulator of force . w
    const int32_t* nbr;
    const uint32_t* bits;      // frozen bond flags
    const int32_t* sw;
    int32_t Q;
    int32_t uniform_w;         // 1: every node has volume vol0
    int64_t n;
    const uint8_t* bcc;
    const BcClass* bct;
    double dt_rho, damp, inv_delta, vol0;
};

cudaError_t launch_adj_mask_publish_dw(const double* ub, const double* vb, const uint8_t* bcc,
                                       const BcClass* bct, double dt, double ws,
                                       const float4* fwd, const double* un, const double* vol,
                                       int64_t n_pad, double inv_delta, double* ubm, double* w,
                                       float4* rec, float4* wrec, cudaStream_t s);
cudaError_t launch_adj_step_dw(const AdjDwArgs& a, int grid, int block, cudaStream_t s);
cudaError_t launch_adj_merge_dw(const float2* acc, int64_t count, double scale, double* gc,
                                cudaStream_t s);

cudaError_t launch_adj_mask(const double* ub, const double* vb, const uint8_t* bcc,
                            const BcClass* bct, int64_t n, double dt, double ws, double* ubm,
                            double* w, cudaStream_t s);
cudaError_t launch_adj_step(const AdjArgs& a, int grid, int block, cudaStream_t s);
cudaError_t launch_extract_u(const double* rec, int64_t n, double* u, cudaStream_t s);
cudaError_t launch_insert_u(const double* u, int64_t n, double* rec, cudaStream_t s);
cudaError_t launch_to_lib3(const double* in, const int32_t* gid, int64_t n, double* out,
                           cudaStream_t s);
cudaError_t launch_from_lib3(const double* in, const int32_t* gid, int64_t n, double* out,
                             cudaStream_t s);
// val (one double per SELL slot) -> out (per directed bond, canonical order);
// off/idx: the canonical family on the device
cudaError_t launch_slots_to_canonical(const double* val, const int32_t* nbr, const int32_t* gid,
                                      const int64_t* off, const int32_t* idx, int64_t n, int Q,
                                      double* out, cudaStream_t s);
// deterministic two-pass sum: out = scale * sum(x[0..n)); partial holds n_partial doubles
int sum_partials_needed(int64_t n);
cudaError_t launch_sum(const double* x, int64_t n, double scale, double* partial, int n_partial,
                       double* out, cudaStream_t s);

// ---- step kernels (pd_step_f32.cu / pd_step_f64.cu) --------------------------
cudaError_t launch_step_f32(const StepArgsF32& a, int sc_mode, int grid, int block,
                            cudaStream_t s);
cudaError_t launch_step_f64(const StepArgsF64& a, int sc_mode, int grid, int block,
                            cudaStream_t s);
const void* step_f32_kernel(int sc_mode, bool uniform_w, bool per_bond_c);
// extended-epilogue build (velocity-Verlet, smooth loading start, force pass)
cudaError_t launch_step_f32_ext(const StepArgsF32& a, int sc_mode, int grid, int block,
                                cudaStream_t s);
const void* step_f32_kernel_ext(int sc_mode, bool uniform_w, bool per_bond_c);
// regular-lattice stencil build of the FP32 Euler-Cromer step (pd_step_f32_lat.cu):
// published records with a zero halo on both sides
cudaError_t launch_step_f32_lat(const StepArgsF32& a, int sc_mode, int grid, int block,
                                cudaStream_t s);
const void* step_f32_kernel_lat(int sc_mode, bool per_bond_c);
// the same for a batch of lattice models (pd_step_f32_lat_batch.cu)
cudaError_t launch_step_f32_lat_batch(const StepArgsF32& a, int sc_mode, int grid, int block,
                                      cudaStream_t s);
const void* step_f32_kernel_lat_batch(int sc_mode, bool per_bond_c);
// both allocated for 3 resident blocks (80 registers; pd_step_f32_lat_r80.cu,
// pd_step_f32_lat_batch_r80.cu), the autotuner's compiled alternative
cudaError_t launch_step_f32_lat_r80(const StepArgsF32& a, int sc_mode, int grid, int block,
                                    cudaStream_t s);
const void* step_f32_kernel_lat_r80(int sc_mode, bool per_bond_c);
cudaError_t launch_step_f32_lat_batch_r80(const StepArgsF32& a, int sc_mode, int grid, int block,
                                          cudaStream_t s);
const void* step_f32_kernel_lat_batch_r80(int sc_mode, bool per_bond_c);
// bilinear-softening build of the FP32 step kernel (pd_step_f32_soft.cu)
cudaError_t launch_step_f32_soft(const StepArgsF32& a, int sc_mode, int grid, int block,
                                 cudaStream_t s);
const void* step_f32_kernel_soft(int sc_mode, bool uniform_w, bool per_bond_c);
const void* step_f64_kernel(int sc_mode);
cudaError_t launch_step_dw(const StepArgsF64& a, const DwArgs& d, int sc_mode, int grid, int block,
                           cudaStream_t s);
const void* step_dw_kernel(int sc_mode, bool uniform_w, bool soft, bool vv);
// double-word records from the FP64 records (positions relative to origin[3])
cudaError_t launch_dw_publish(const double* rec64, float4* rec, int64_t n_pad, const double* origin,
                              double inv_delta, cudaStream_t s);
// every slot's |xi| / delta (1 where there is no bond)
cudaError_t launch_dw_len(const double* x64, const int32_t* nbr, int64_t n, int Q,
                          double inv_delta, float2* len, cudaStream_t s);
// double-word copy of an FP64 per-slot array
cudaError_t launch_dw_split(const double* in, int64_t count, float2* out, cudaStream_t s);

// ---- helper kernels (pd_aux.cu) ---------------------------------------------
cudaError_t launch_advance(int64_t* step_ctr, int64_t k, cudaStream_t s);
// caller-order FP64 (u, v) <-> internal state; u_out/v_out/u_in/v_in may be null
cudaError_t launch_get_state_f32(const float4* rec, const float4* lo32, const float* v32,
                                 const int32_t* gid, int64_t n, double delta, double* u_out,
                                 double* v_out, cudaStream_t s);
cudaError_t launch_set_state_f32(const double* u_in, const double* v_in, const int32_t* gid,
                                 int64_t n, double inv_delta, float4* rec, float4* lo32,
                                 float* v32, cudaStream_t s);
// regular-lattice FP32 models: FP64 displacement (in units of delta, or of each
// instance's spacing in a batch: inst / itab non-null) and FP32 velocity
cudaError_t launch_get_state_lat(const double* u_lat, const float* v32, const int32_t* gid,
                                 int64_t n, double delta, const int32_t* inst,
                                 const InstParams* itab, double* u_out, double* v_out,
                                 cudaStream_t s);
cudaError_t launch_set_state_lat(const double* u_in, const double* v_in, const int32_t* gid,
                                 int64_t n, double inv_delta, const int32_t* inst,
                                 const InstParams* itab, double* u_lat, float4* pub, float* v32,
                                 cudaStream_t s);
cudaError_t launch_get_state_f64(const double* rec64, const double* v64, const int32_t* gid,
                                 int64_t n, double* u_out, double* v_out, cudaStream_t s);
cudaError_t launch_set_state_f64(const double* u_in, const double* v_in, const int32_t* gid,
                                 int64_t n, double* rec64, double* v64, cudaStream_t s);
// damage from the bond flags (Eq. 8), written to caller order
// (integ: per-slot integrity weighting each intact bond, or nullptr)
cudaError_t launch_damage(int precision, const void* wrec, const int32_t* nbr,
                          const uint32_t* bits, const int32_t* sw, const void* wsum_inv,
                          const int32_t* gid, int64_t n, int Q, const void* integ,
                          double* phi_out, cudaStream_t s);
// flag |= 1 if any of x[0..m) is not finite
cudaError_t launch_check_finite(const double* x, int64_t m, int* flag, cudaStream_t s);
// clear the bond flags of m slots (bits[word[e]] &= ~mask[e]) and zero their
// integrity when integ is not null (float for precision 32, else double)
cudaError_t launch_clear_slots(uint32_t* bits, const int64_t* word, const uint32_t* mask,
                               const int64_t* slot, int64_t m, int precision, void* integ,
                               cudaStream_t s);
// fill n values of `precision` (32 or 64) with v
cudaError_t launch_fill(int precision, void* dst, int64_t n, double v, cudaStream_t s);
// damage written by the last step -> caller order
cudaError_t launch_gather_damage(int precision, const void* dmg, const int32_t* gid, int64_t n,
                                 double* phi_out, cudaStream_t s);
// node weights w = wscale * V (FP32: the w array, passed as wrec0; FP64: both
// record buffers) and wsum_inv (a slot is a real member iff its init_bits bit is set)
// state-based model: per-slot |xi| and weighted volumes (once), and one step
// (dilation kernel, then force + integration kernel)
cudaError_t launch_osb_setup(const StepArgsF64& a, const OsbArgs& o, const double* x64,
                             cudaStream_t s);
cudaError_t launch_osb_step(const StepArgsF64& a, const OsbArgs& o, int grid, int block,
                            cudaStream_t s);
cudaError_t launch_osb32_setup(const StepArgsF32& a, const OsbArgs32& o, cudaStream_t s);
// the two state-based launches, each on a grid sized by its own occupancy
cudaError_t launch_osb32_step(const StepArgsF32& a, const OsbArgs32& o, int sc_mode, int grid,
                              int grid_dil, int block, cudaStream_t s);
const void* osb32_dilation_kernel(int sc_mode, bool uniform_w);
const void* osb32_force_kernel(int sc_mode, bool uniform_w);
// per slot 1 / |x_j - x_i| from the FP64 reference positions (0 for unused slots)
cudaError_t launch_inv_len(const double* x64, const int32_t* nbr, const int32_t* sw, int64_t n,
                           int Q, double* ilen, cudaStream_t s);
// step_ctr[0] is the device step counter; step_ctr[1] the step at which the
// state was last set (velocity-Verlet forms a^n afresh there)

#ifdef __CUDACC__
// Displacement scale after step k: rate * k, or with a smooth start over T
// steps (a fifth-order displacement-time curve, zero initial velocity and
// acceleration): rate * T * P(k/T), P(t) = t^4 - (3/5) t^5, then the line
// rate * (k - 3T/5) that continues it.
__device__ __forceinline__ double bc_scale(double rate, int64_t T, int64_t k)
{
    if (T <= 0) return rate * (double)k;
    if (k >= T) return rate * ((double)k - 0.6 * (double)T);
    const double t = (double)k / (double)T;
    return rate * (double)T * (t * t * t * t - 0.6 * t * t * t * t * t);
}
#endif

#ifdef __CUDACC__
// Softening integrity mu = envelope(s) / (c s) for s_0 < s < s_c: bilinear (the
// force falls linearly from c s_0 to 0 at s_c) or, with k1 > 1, trilinear (from
// c s_0 to beta c s_0 at the kink s_1 = k1 s_0, then to 0 at s_c)
__device__ __forceinline__ double soft_mu_of(double s, double s0, double sc, double k1,
                                             double beta)
{
    if (k1 > 1.0) {
        const double s1 = k1 * s0;
        if (s <= s1) return s0 * ((1.0 - beta) * (s1 - s) / (s1 - s0) + beta) / s;
        return s0 * beta * (sc - s) / ((sc - s1) * s);
    }
    return s0 * (sc - s) / (s * (sc - s0));
}
#endif

// 1/sqrt(x), x > 0, in FP64: the FP32 hardware estimate refined by two
// Newton-Raphson steps for f(y) = 1/y^2 - x (quadratic convergence: relative
// error ~2^-22 -> ~2^-43 -> rounding level); residual r = 1 - x y^2 taken with
// a fused multiply-add, y <- y + (y/2) r.  Outside the FP32 range of the
// estimate it falls back to 1/sqrt(x).
#ifdef __CUDACC__
__device__ __forceinline__ double rsqrt_nr(double x)
{
    const float xf = (float)x;
    if (!(xf > 0.0f) || isinf(xf)) return 1.0 / sqrt(x);
    double y = (double)rsqrtf(xf);
    double t = x * y;
    y = fma(0.5 * y, fma(-t, y, 1.0), y);
    t = x * y;
    y = fma(0.5 * y, fma(-t, y, 1.0), y);
    return y;
}
#endif
cudaError_t launch_set_weights(int precision, void* wrec0, void* wrec1, const double* vol,
                               const int32_t* nbr, const uint32_t* init_bits, const int32_t* sw,
                               int64_t n, int Q, double wscale, void* wsum_inv, cudaStream_t s);

}  // namespace pd
