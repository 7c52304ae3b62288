// C ABI of the peridynamic step library: handle lifecycle, step orchestration
// (direct launches or captured CUDA graphs of `graph_steps` steps driven by a
// device step counter), state transfer and parameter updates.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "../../include/pd.h"
#include "pd_internal.h"
#include "pd_prep.h"

namespace {
// NVTX range around each public entry point (a no-op unless a profiler is
// attached): profiles and ncu's --nvtx filters see the calls by name.
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};
}  // namespace

using namespace pd;

namespace {

thread_local std::string g_err;

// relative band around s_c within which the FP32 path re-tests bonds in FP64
constexpr double kGuard = 5e-4;

pd_status fail(pd_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

pd_status cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(PD_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(PD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define PD_CUDA(call, what)                                \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

bool finite_all(const double* p, int64_t m)
{
    for (int64_t i = 0; i < m; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

struct pd_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int precision = 64;
    int Q = 1;
    int64_t n = 0, n_pad = 0, n_slices = 0, n_bonds = 0;
    double delta = 0, dt = 0, eta = 0, rho = 0;
    double c = 0, sc = 0, sc_lo = 0, sc_hi = 0;
    int sc_mode = 0;
    uint64_t sc_seed = 0;
    double disp_rate = 0, load = 0;
    bool has_nofail = false;
    bool per_bond_c = false;
    int64_t step = 0;
    int graph_steps = 0;
    cudaGraphExec_t graph = nullptr;
    int grid = 0, block = 256, blocks_per_sm = 0;
    bool damage_fresh = false;

    std::vector<int64_t> off;  // canonical family after cuts
    std::vector<int32_t> idx;
    std::vector<int32_t> perm, inv, cnt;

    std::vector<void*> allocs;
    int64_t device_bytes = 0;
    // FP32 path: 2 float4 per node (+ owner-private lo, weights); FP64: 8 doubles per node
    float4* rec32[2] = {nullptr, nullptr};
    float4* lo32 = nullptr;
    float* w32 = nullptr;
    bool uniform_vol = false;
    double vol0 = 0.0;
    double* rec[2] = {nullptr, nullptr};
    // both
    void* v = nullptr;
    int32_t* nbr = nullptr;
    uint32_t* bits = nullptr;
    uint32_t* bits0 = nullptr;  // bond flags after the initial cuts
    int32_t* sw = nullptr;
    void* cbond = nullptr;
    uint8_t* bcc = nullptr;
    BcClass* bct = nullptr;
    int32_t* gid = nullptr;
    double* x64 = nullptr;
    double* vol = nullptr;
    double* ilen = nullptr;  // FP64: per slot 1 / |xi|
    // PD_PREC_DW: FP64 layout and integration, bonds in double-word FP32 arithmetic
    bool dw = false;
    float4* recdw[2] = {nullptr, nullptr};  // double-word copies of the records
    float2* lendw = nullptr;                // per slot |xi| / delta
    float2* cbdw = nullptr;                 // per slot c_ij (per-bond stiffness)
    double dw_origin[3] = {0.0, 0.0, 0.0};  // origin of the double-word positions
    int integrator = PD_INTEGRATOR_EC;
    int64_t ramp_steps = 0;
    void* vpeek = nullptr;  // velocity-Verlet: full-step velocity for pd_get_state
    int64_t peek_step = -1; // step whose force pass filled vpeek (-1: none)
    int64_t vv_start = 0;   // step of the last set state (velocity-Verlet: a^n formed afresh)
    int grid_dil = 0;       // grids of the FP32 state-based dilation and force kernels
    int grid_osbf = 0;
    double kr = 0.0;        // >= 1: bilinear softening, s_0 = s_c / kr
    double k1 = 0.0, beta = 1.0;  // trilinear kink (k1 > 1)
    void* integ = nullptr;  // softening: per-slot integrity (float / double)
    int model = 0;          // 1: ordinary state-based linear solid (FP64)
    double osb_K = 0.0, osb_G = 0.0;
    double* osb_len = nullptr;    // per slot |xi|
    double* osb_mvol = nullptr;   // per node weighted volume
    double* osb_theta = nullptr;  // per node dilation
    double* osb_alpha = nullptr;  // per node force-scalar coefficients (see pd_step_osb.cu)
    double* osb_beta = nullptr;
    float4* osbdw_ab = nullptr;   // double-word state-based: per node alpha~, beta~
    float *osb32_mvol = nullptr, *osb32_theta = nullptr;  // FP32 state-based arrays
    float2* osb32_ab = nullptr;
    float4* osblat_coef = nullptr;  // FP32 state-based lattice models (pd_step_f32_lat_osb.cu)
    float4* osblat_rec = nullptr;
    float* osblat_b = nullptr;
    uint8_t* osblat_exact = nullptr;
    void* wsum_inv = nullptr;
    void* damage = nullptr;
    int* err = nullptr;
    int64_t* step_ctr = nullptr;
    double* staging = nullptr;  // 3n doubles for host transfers
    // adjoint: frozen bond flags during its forward runs, and the recorded run
    bool frozen = false;
    struct Tape {
        bool valid = false;
        bool vv = false;  // velocity-Verlet run (opens with a half kick, ends with one)
        int64_t N = 0, C = 0, nck = 0, step0 = 0;
        double *ck_u = nullptr, *ck_v = nullptr, *seg = nullptr, *fin_u = nullptr,
               *fin_v = nullptr;
        int64_t cap_ck = 0, cap_seg = 0;
        double *ub[2] = {nullptr, nullptr}, *vb[2] = {nullptr, nullptr}, *ubm = nullptr,
               *w = nullptr, *gc = nullptr, *gl = nullptr, *partial = nullptr, *out = nullptr;
        int n_partial = 0;
        // double-word reverse sweep (PD_PREC_DW): records of u^n and w, and the
        // per-slot gradient accumulator
        float4 *rrec = nullptr, *wrec = nullptr;
        float2* gcdw = nullptr;
    } tape;
    // regular lattice (FP32 Euler-Cromer PMB models): stencil-ordered layout,
    // FP64 displacement and FP32 published records with a halo of lat_halo
    // records on both sides (no rec32 / lo32)
    bool lattice = false;
    std::vector<Lattice> lats;      // one per instance (a single model: one)
    std::vector<int32_t> lat_of;    // batches: the lattice of each library position
    int64_t lat_halo = 0;
    int lat_var = 0;                // the stencil step's variant (pd_config.lat_variant)
    LatTmaArgs lat_tma{};           // variants 2..4: the tile copies' tensor maps and tiling
    int lat_tma_shape = -1;         // the box shape lat_tma holds maps for
    double* lat_u[2] = {nullptr, nullptr};   // u / delta, FP64, 3 per node
    float4* lat_pub[2] = {nullptr, nullptr}; // FP32 copies the neighbours read
    // batches: instance of each node, instance-local ids, per-instance s_c table
    bool batch = false;
    std::vector<int64_t> inst_off;
    int32_t* inst = nullptr;
    int32_t* hid = nullptr;
    InstParams* itab = nullptr;

    template <class T>
    cudaError_t alloc(T** p, size_t count)
    {
        void* q = nullptr;
        const size_t bytes = std::max<size_t>(count * sizeof(T), 256);
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) return e;
        allocs.push_back(q);
        device_bytes += (int64_t)bytes;
        *p = (T*)q;
        return cudaMemsetAsync(q, 0, bytes, stream);
    }

    void release()
    {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
        if (stream) cudaStreamSynchronize(stream);
        for (void* p : allocs) cudaFree(p);
        allocs.clear();
        if (own_stream && stream) cudaStreamDestroy(stream);
        stream = nullptr;
    }

    void drop_graph()
    {
        if (graph) cudaGraphExecDestroy(graph);
        graph = nullptr;
    }

    const void* wrec() const
    {
        return precision == 32 ? (const void*)w32 : (const void*)rec[0];
    }
};

namespace {

StepArgsF32 args_f32(pd_handle* h, int k, int64_t step_abs = -1)
{
    StepArgsF32 a{};
    a.inst = h->inst;
    a.itab = h->itab;
    a.hid = h->hid;
    a.rec[0] = h->rec32[0];
    a.rec[1] = h->rec32[1];
    a.lo32 = h->lo32;
    a.w = h->w32;
    a.uniform_w = h->uniform_vol ? 1 : 0;
    a.w_const = (float)(((h->per_bond_c || h->model == 1) ? 1.0 : h->c) * h->vol0);
    a.v = (float*)h->v;
    a.nbr = h->nbr;
    a.bits = h->bits;
    a.sw = h->sw;
    a.cbond = h->per_bond_c ? (const float*)h->cbond : nullptr;
    a.bcc = h->bcc;
    a.bct = h->bct;
    a.gid = h->gid;
    a.x64 = h->x64;
    a.wsum_inv = (const float*)h->wsum_inv;
    a.damage = (float*)h->damage;
    a.err = h->err;
    a.step_ctr = h->step_ctr;
    a.n = h->n;
    a.k = k;
    a.step_abs = h->lattice ? step_abs : -1;
    a.Q = h->Q;
    a.has_nofail = h->has_nofail ? 1 : 0;
    a.guard = (float)kGuard;
    a.sc_f = (float)h->sc;
    a.sc_lo_f = (float)h->sc_lo;
    a.fast_lo = (float)((1.0 - 2.0 * a.guard) * h->sc_lo);
    if (h->integ != nullptr) {  // softening: the band below the smallest s_0 is resolved too
        a.integ = (float*)h->integ;
        a.kr = h->kr;
        a.k1 = h->k1;
        a.beta = h->beta;
        a.fast_lo = (float)((1.0 - 2.0 * a.guard) * h->sc_lo / h->kr);
    }
    a.sc = h->sc;
    a.sc_lo = h->sc_lo;
    a.sc_hi = h->sc_hi;
    a.sc_seed = h->sc_seed;
    a.dt = h->dt;
    a.eta = h->eta;
    a.rho = h->rho;
    a.disp_rate = h->disp_rate;
    a.load = h->load;
    a.ramp_steps = h->ramp_steps;
    a.vv = h->integrator == PD_INTEGRATOR_VV ? 1 : 0;
    a.delta = h->delta;
    a.inv_delta = 1.0 / h->delta;
    a.dt_f = (float)h->dt;
    a.eta_f = (float)h->eta;
    a.rho_f = (float)h->rho;
    a.dtd_f = (float)(a.dt * a.inv_delta);
    if (h->lattice) {
        a.lat_u[0] = h->lat_u[0];
        a.lat_u[1] = h->lat_u[1];
        a.lat_pub[0] = h->lat_pub[0];
        a.lat_pub[1] = h->lat_pub[1];
        // a single model in horizon units; a batch in each instance's lattice
        // units (kappa = 1; strides and thresholds per instance in itab)
        a.lat_sy = h->batch ? 0 : (int32_t)h->lats[0].N[2];
        a.lat_sx = h->batch ? 0 : (int32_t)(h->lats[0].N[1] * h->lats[0].N[2]);
        const double kap = h->batch ? 1.0 : h->lats[0].dx / h->delta;
        const double f = (1.0 - 2.0 * kGuard) * h->sc_lo;
        for (int c = -3; c <= 3; ++c) {
            a.lat_xi[c + 3] = (float)(kap * c);
            a.lat_xi2[c + 3] = 2.0f * a.lat_xi[c + 3];
        }
        for (int j = 0; j < kStencilRows; ++j) {
            const Off3 r = stencil_row(j);
            a.lat_rxi[j] = make_float4(a.lat_xi[r.x + 3], a.lat_xi[r.y + 3], a.lat_xi2[r.x + 3],
                                       a.lat_xi2[r.y + 3]);
            a.lat_roff[j] = r.x * a.lat_sx + r.y * a.lat_sy;
            a.lat_rox[j] = r.x;
            a.lat_roy[j] = r.y;
        }
        for (int j = 0; j + 1 < kStencilRows; ++j) {
            const Off3 r0 = stencil_row(j), r1 = stencil_row(j + 1);
            a.lat_rxp[j][0] = make_float4(a.lat_xi[r0.x + 3], a.lat_xi[r1.x + 3],
                                          a.lat_xi[r0.y + 3], a.lat_xi[r1.y + 3]);
            a.lat_rxp[j][1] = make_float4(a.lat_xi2[r0.x + 3], a.lat_xi2[r1.x + 3],
                                          a.lat_xi2[r0.y + 3], a.lat_xi2[r1.y + 3]);
        }
        for (int q = 0; q <= kStencilR2; ++q) {
            a.lat_q[q] = (float)(kap * kap * q);
            a.lat_l[q] = (float)(kap * std::sqrt((double)q));
            a.lat_thr[q] = (float)(f * (2.0 + f) * kap * kap * q);
            if (q == 0) continue;  // no stencil offset
            // num / D = num g(x) / |xi|^3 with g = 1/2 - 3x/8 + 5x^2/16 + O(x^3), x = num / |xi|^2
            const double qq = kap * kap * q, L = kap * std::sqrt((double)q);
            a.lat_pc[0][q] = (float)(0.5 / (L * qq));
            a.lat_pc[1][q] = (float)(-0.375 / (L * qq * qq));
            a.lat_pc[2][q] = (float)(0.3125 / (L * qq * qq * qq));
            // |xi| e~ = num (1/2 - x/8 + x^2/16 + O(x^3)) for the state-based dilation
            a.lat_dc[0][q] = 0.5f;
            a.lat_dc[1][q] = (float)(-0.125 / qq);
            a.lat_dc[2][q] = (float)(0.0625 / (qq * qq));
            const double pt = kLatPolyX * qq, tu = std::min(f * (2.0 + f) * qq, pt);
            a.lat_pt[q] = (float)pt;
            a.lat_cc[q] = (float)(0.5 * (tu - pt));
            a.lat_ch[q] = (float)(0.5 * (tu + pt));
            for (int t = 0; t < 3; ++t) {
                a.lat_pcd[t][q] = make_float2(a.lat_pc[t][q], a.lat_pc[t][q]);
                a.lat_dcd[t][q] = make_float2(a.lat_dc[t][q], a.lat_dc[t][q]);
            }
            a.lat_ccd[q] = make_float2(-a.lat_cc[q], -a.lat_cc[q]);
            // (1 + x)^(-1/2) = 1 - x/2 + 3x^2/8 + O(x^3); 1 - (1 + x)^(-1/2) = x/2 - 3x^2/8
            // + 5x^3/16 + O(x^4), x = num / |xi|^2
            const float fa[2] = {(float)(-0.5 / qq), (float)(0.375 / (qq * qq))};
            const float fb[3] = {(float)(0.5 / qq), (float)(-0.375 / (qq * qq)),
                                 (float)(0.3125 / (qq * qq * qq))};
            for (int t = 0; t < 3; ++t) {
                if (t < 2) a.lat_fad[t][q] = make_float2(fa[t], fa[t]);
                a.lat_fbd[t][q] = make_float2(fb[t], fb[t]);
            }
        }
    }
    return a;
}

StepArgsF64 args_f64(pd_handle* h, int k)
{
    StepArgsF64 a{};
    a.inst = h->inst;
    a.itab = h->itab;
    a.hid = h->hid;
    a.rec[0] = h->rec[0];
    a.rec[1] = h->rec[1];
    a.v = (double*)h->v;
    a.nbr = h->nbr;
    a.bits = h->bits;
    a.sw = h->sw;
    a.cbond = h->per_bond_c ? (const double*)h->cbond : nullptr;
    a.ilen = h->ilen;
    a.integ = (double*)h->integ;
    a.kr = h->kr;
    a.k1 = h->k1;
    a.beta = h->beta;
    a.bcc = h->bcc;
    a.bct = h->bct;
    a.gid = h->gid;
    a.wsum_inv = (const double*)h->wsum_inv;
    a.damage = (double*)h->damage;
    a.err = h->err;
    a.step_ctr = h->step_ctr;
    a.n = h->n;
    a.k = k;
    a.Q = h->Q;
    a.has_nofail = h->has_nofail ? 1 : 0;
    a.frozen = h->frozen ? 1 : 0;
    a.sc = h->sc;
    a.sc_lo = h->sc_lo;
    a.sc_hi = h->sc_hi;
    a.sc_seed = h->sc_seed;
    a.dt = h->dt;
    a.eta = h->eta;
    a.rho = h->rho;
    a.disp_rate = h->disp_rate;
    a.load = h->load;
    a.ramp_steps = h->ramp_steps;
    a.vv = h->integrator == PD_INTEGRATOR_VV ? 1 : 0;
    return a;
}

// the FP32 step kernel build for this handle (bilinear softening or not)
cudaError_t launch_f32(pd_handle* h, const StepArgsF32& a)
{
    // a regular-lattice model (created only for the Euler-Cromer PMB step with a
    // linear loading ramp and uniform volumes) has the stencil kernel's state
    if (h->lattice && h->lat_var >= 2)
        return launch_step_f32_lat_tma(a, h->lat_tma, h->lat_var - 2, h->sc_mode, h->grid,
                                       h->stream);
    if (h->lattice && h->batch)
        return h->lat_var == 1
                   ? launch_step_f32_lat_batch_r80(a, h->sc_mode, h->grid, h->block, h->stream)
                   : launch_step_f32_lat_batch(a, h->sc_mode, h->grid, h->block, h->stream);
    if (h->lattice)
        return h->lat_var == 1
                   ? launch_step_f32_lat_r80(a, h->sc_mode, h->grid, h->block, h->stream)
                   : launch_step_f32_lat(a, h->sc_mode, h->grid, h->block, h->stream);
    if (h->integ != nullptr) return launch_step_f32_soft(a, h->sc_mode, h->grid, h->block, h->stream);
    if (a.vv || a.ramp_steps > 0 || a.peek)
        return launch_step_f32_ext(a, h->sc_mode, h->grid, h->block, h->stream);
    return launch_step_f32(a, h->sc_mode, h->grid, h->block, h->stream);
}

const void* f32_kernel(pd_handle* h)
{
    if (h->lattice && h->lat_var >= 2)
        return step_f32_kernel_lat_tma(h->lat_var - 2, h->sc_mode, h->per_bond_c);
    if (h->lattice && h->batch)
        return h->lat_var == 1 ? step_f32_kernel_lat_batch_r80(h->sc_mode, h->per_bond_c)
                               : step_f32_kernel_lat_batch(h->sc_mode, h->per_bond_c);
    if (h->lattice)
        return h->lat_var == 1 ? step_f32_kernel_lat_r80(h->sc_mode, h->per_bond_c)
                               : step_f32_kernel_lat(h->sc_mode, h->per_bond_c);
    return h->integ != nullptr ? step_f32_kernel_soft(h->sc_mode, h->uniform_vol, h->per_bond_c)
                               : step_f32_kernel(h->sc_mode, h->uniform_vol, h->per_bond_c);
}

OsbArgs osb_args(pd_handle* h)
{
    OsbArgs o{};
    o.len = h->osb_len;
    o.vol = h->vol;
    o.mvol = h->osb_mvol;
    o.theta = h->osb_theta;
    o.alpha = h->osb_alpha;
    o.beta = h->osb_beta;
    o.K = h->osb_K;
    o.G = h->osb_G;
    return o;
}

OsbDwArgs osbdw_args(pd_handle* h)
{
    OsbDwArgs o{};
    o.len = h->lendw;
    o.vol = h->vol;
    o.mvol = h->osb_mvol;
    o.theta = h->osb_theta;
    o.ab = h->osbdw_ab;
    o.K = h->osb_K;
    o.G = h->osb_G;
    return o;
}

OsbLatArgs osblat_args(pd_handle* h)
{
    OsbLatArgs o{};
    o.coef = h->osblat_coef;
    o.rec = h->osblat_rec;
    o.bco = h->osblat_b;
    o.theta = h->osb32_theta;
    o.exact = h->osblat_exact;
    return o;
}

OsbArgs32 osb32_args(pd_handle* h)
{
    OsbArgs32 o{};
    o.mvol = h->osb32_mvol;
    o.theta = h->osb32_theta;
    o.ab = h->osb32_ab;
    o.K = h->osb_K;
    o.G = h->osb_G;
    o.delta = h->delta;
    return o;
}

DwArgs dw_args(pd_handle* h)
{
    DwArgs d{};
    d.rec[0] = h->recdw[0];
    d.rec[1] = h->recdw[1];
    d.len = h->lendw;
    d.cb = h->per_bond_c ? h->cbdw : nullptr;
    d.inv_delta = 1.0 / h->delta;
    d.w_const = ((h->per_bond_c || h->model == 1) ? 1.0 : h->c) * h->vol0;
    d.dt_rho = h->dt / h->rho;
    // the leading word of a double-word stretch is within 2^-23 of it: below
    // this band the break test cannot be near any s_c of the model
    // (with softening: below the smallest s_0 = s_c / kr)
    d.fast_lo = h->frozen ? INFINITY
                          : (float)((1.0 - 0x1.0p-20) * (h->sc_mode == 0 ? h->sc : h->sc_lo) /
                                    (h->integ != nullptr ? h->kr : 1.0));
    // batches: the per-node weights (each instance's c folded in)
    d.uniform_w = h->uniform_vol && !h->batch ? 1 : 0;
    return d;
}

// double-word records of both buffers from the FP64 records
pd_status dw_publish(pd_handle* h)
{
    if (!h->dw) return PD_OK;
    for (int b = 0; b < 2; ++b)
        PD_CUDA(launch_dw_publish(h->rec[b], h->recdw[b], h->n_pad, h->dw_origin, 1.0 / h->delta,
                                  h->stream),
                "double-word records");
    return PD_OK;
}

const void* step_kernel_fn(pd_handle* h)
{
    if (h->precision == 32) return f32_kernel(h);
    if (h->dw)
        return step_dw_kernel(h->sc_mode, h->uniform_vol && !h->batch, h->integ != nullptr,
                              h->integrator == PD_INTEGRATOR_VV);
    return step_f64_kernel(h->sc_mode);
}

// One step launch, k steps past the device counter; step_abs >= 0 (F32 lattice
// handles, direct launches): the absolute step, the kernel then advancing the
// counter itself
cudaError_t launch_one(pd_handle* h, int k, int64_t step_abs = -1)
{
    if (h->dw && h->model == 1)
        return launch_osb_dw_step(args_f64(h, k), dw_args(h), osbdw_args(h), h->grid, h->block,
                                  h->stream);
    if (h->dw)
        return launch_step_dw(args_f64(h, k), dw_args(h), h->sc_mode, h->grid, h->block,
                              h->stream);
    if (h->model == 1 && h->precision == 32)
        return h->lattice
                   ? launch_osb_lat_step(args_f32(h, k, step_abs), osblat_args(h), h->sc_mode, h->grid,
                                         h->grid_osbf, h->block, h->stream)
                   : launch_osb32_step(args_f32(h, k), osb32_args(h), h->sc_mode, h->grid_osbf, h->grid_dil, h->block,
                                 h->stream);
    if (h->model == 1)
        return launch_osb_step(args_f64(h, k), osb_args(h), h->grid, h->block, h->stream);
    if (h->precision == 32)
        return launch_f32(h, args_f32(h, k, step_abs));
    return launch_step_f64(args_f64(h, k), h->sc_mode, h->grid, h->block, h->stream);
}

// The tensor maps of the tile step's copies (both record buffers) for box shape
// `shape`, and its tiling of the lattice.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

pd_status encode_lat_tma(pd_handle* h, int shape)
{
    if (h->lat_tma_shape == shape) return PD_OK;
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(PD_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        encode = (EncodeTiledFn)fn;
    }
    const Lattice& L = h->lats[0];
    const int64_t nx = L.N[0], ny = L.N[1], nz = L.N[2];
    const int bz = lat_tma_dim(shape, 0), by = lat_tma_dim(shape, 1), bx = lat_tma_dim(shape, 2);
    LatTmaArgs t{};
    t.nz = (int32_t)nz;
    t.ny = (int32_t)ny;
    t.nx = (int32_t)nx;
    t.tiles_z = (int32_t)((nz + bz - 1) / bz);
    t.tiles_y = (int32_t)((ny + by - 1) / by);
    t.tiles_x = (int32_t)((nx + bx - 1) / bx);
    t.extra_tx = h->lat_tma.extra_tx;
    // records {x, y, z, 0} of node (ix Ny + iy) Nz + iz: the innermost dimension
    // is the record's 4 floats (16 bytes), then z, y, x
    const cuuint64_t dims[4] = {4, (cuuint64_t)nz, (cuuint64_t)ny, (cuuint64_t)nx};
    const cuuint64_t strides[3] = {16, (cuuint64_t)(16 * nz), (cuuint64_t)(16 * nz * ny)};
    const cuuint32_t box[4] = {4, (cuuint32_t)(bz + 6), (cuuint32_t)(by + 6), (cuuint32_t)(bx + 6)};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int k = 0; k < 2; ++k) {
        const CUresult r =
            encode(&t.map[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void*)h->lat_pub[k], dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(PD_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    h->lat_tma = t;
    h->lat_tma_shape = shape;
    return PD_OK;
}

pd_status choose_grid(pd_handle* h, int blocks_per_sm)
{
    if (h->lattice && h->lat_var >= 2) {  // the tile step: one block per box of the lattice
        const int shape = h->lat_var - 2;
        pd_status st = encode_lat_tma(h, shape);
        if (st != PD_OK) return st;
        const void* fn = step_kernel_fn(h);
        PD_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)lat_tma_smem_bytes(shape)),
                "shared memory size");
        PD_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared),
                "carveout");
        h->block = lat_tma_dim(shape, 0) * lat_tma_dim(shape, 1) * lat_tma_dim(shape, 2);
        const int64_t tiles = (int64_t)h->lat_tma.tiles_z * h->lat_tma.tiles_y * h->lat_tma.tiles_x;
        if (tiles > 0x7fffffff) return fail(PD_ERR_ARG, "lattice too large for the tile step");
        h->grid = (int)tiles;
        h->grid_dil = h->grid;
        h->grid_osbf = h->grid;
        return PD_OK;
    }
    int sms = 0;
    PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device), "sm count");
    const void* fn = step_kernel_fn(h);
    // no shared memory is used: give the unified L1/shared array to L1
    PD_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 0),
            "carveout");
    int occ = 0;
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, h->block, 0), "occupancy");
    if (occ < 1) occ = 1;
    if (blocks_per_sm > 0) occ = std::min(occ, blocks_per_sm);
    const int64_t warps_per_block = h->block / 32;
    const int64_t need = (h->n_slices + warps_per_block - 1) / warps_per_block;
    h->grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * occ, need));
    h->grid_dil = h->grid;
    h->grid_osbf = h->grid;
    if (h->model == 1 && h->precision == 32 && h->lattice) {  // the force loop's own grid
        const void* ff = osb_lat_force_kernel();
        PD_CUDA(cudaFuncSetAttribute(ff, cudaFuncAttributePreferredSharedMemoryCarveout, 0),
                "carveout");
        int o = 0;
        PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, ff, h->block, 0), "occupancy");
        if (blocks_per_sm > 0) o = std::min(o, blocks_per_sm);
        h->grid_osbf = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * std::max(o, 1), need));
    }
    if (h->model == 1 && h->precision == 32 && !h->lattice) {  // the state-based kernels' own grids
        auto grid_of_kernel = [&](const void* fn, int& out) -> pd_status {
            PD_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 0),
                    "carveout");
            int o = 0;
            PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, fn, h->block, 0), "occupancy");
            if (blocks_per_sm > 0) o = std::min(o, blocks_per_sm);
            out = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * std::max(o, 1), need));
            return PD_OK;
        };
        pd_status st = grid_of_kernel(osb32_dilation_kernel(h->sc_mode, h->uniform_vol), h->grid_dil);
        if (st == PD_OK)
            st = grid_of_kernel(osb32_force_kernel(h->sc_mode, h->uniform_vol), h->grid_osbf);
        if (st != PD_OK) return st;
    }
    return PD_OK;
}

pd_status upload_weights(pd_handle* h)
{
    // node weights: c V (bond-based), V (per-bond stiffness, state-based)
    const double wscale = (h->per_bond_c || h->model == 1) ? 1.0 : h->c;
    void* w0 = h->precision == 32 ? (void*)h->w32 : (void*)h->rec[0];
    void* w1 = h->precision == 32 ? nullptr : (void*)h->rec[1];
    PD_CUDA(launch_set_weights(h->precision, w0, w1, h->vol, h->nbr, h->bits0, h->sw, h->n, h->Q,
                               wscale, h->wsum_inv, h->stream),
            "set weights");
    return dw_publish(h);
}

pd_status check_dev_err(pd_handle* h)
{
    int e = 0;
    PD_CUDA(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
            "read error flag");
    PD_CUDA(cudaStreamSynchronize(h->stream), "synchronize");
    if (e & PD_DEVERR_NONFINITE)
        return fail(PD_ERR_NONFINITE, "a displacement became non-finite (check dt and loads)");
    if (e & PD_DEVERR_TIMEOUT)
        return fail(PD_ERR_TIMEOUT, "a bounded device wait ran out (the tile copy of the step)");
    return PD_OK;
}

// Velocity-Verlet evaluates the force at u^n at the start of the next step;
// what the method has at the end of step n (the breaks at u^n, the full-step
// velocity v^n) comes from that pass run once ahead: it records the breaks
// (the next step would make the same decisions on the same u^n) and writes
// v^n into vpeek, nothing else.  Cached per step.
pd_status vv_force_pass(pd_handle* h)
{
    if (h->integrator != PD_INTEGRATOR_VV || h->peek_step == h->step) return PD_OK;
    cudaError_t e;
    if (h->precision == 32) {
        StepArgsF32 a = args_f32(h, 0);
        a.peek = 1;
        a.vout = (float*)h->vpeek;
        e = h->model == 1 ? launch_osb32_step(a, osb32_args(h), h->sc_mode, h->grid_osbf, h->grid_dil, h->block,
                                              h->stream)
                          : launch_f32(h, a);
    } else {
        StepArgsF64 a = args_f64(h, 0);
        a.peek = 1;
        a.vout = (double*)h->vpeek;
        if (h->model == 1)
            e = h->dw ? launch_osb_dw_step(a, dw_args(h), osbdw_args(h), h->grid, h->block,
                                           h->stream)
                      : launch_osb_step(a, osb_args(h), h->grid, h->block, h->stream);
        else
            e = h->dw ? launch_step_dw(a, dw_args(h), h->sc_mode, h->grid, h->block, h->stream)
                      : launch_step_f64(a, h->sc_mode, h->grid, h->block, h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "velocity-Verlet force pass");
    h->peek_step = h->step;
    h->damage_fresh = false;  // breaks may have been recorded: damage from the flags
    return PD_OK;
}

// canonical position of every SELL slot, computed on demand from the device family
pd_status canonical_slots(pd_handle* h, std::vector<int64_t>& pos)
{
    std::vector<int32_t> nbr((size_t)(h->n_slices * 32 * h->Q * 32));
    PD_CUDA(cudaStreamSynchronize(h->stream), "synchronize");
    PD_CUDA(cudaMemcpy(nbr.data(), h->nbr, nbr.size() * 4, cudaMemcpyDeviceToHost), "copy family");
    slot_to_canonical(h->n, h->off, h->idx, h->perm, nbr, h->cnt, h->Q, pos);
    return PD_OK;
}

}  // namespace

extern "C" {

const char* pd_last_error(void) { return g_err.c_str(); }

pd_status pd_micromodulus(double K, double delta, double* c_out)
{
    if (!c_out) return fail(PD_ERR_ARG, "c_out is NULL");
    if (!(K > 0.0) || !(delta > 0.0) || !std::isfinite(K) || !std::isfinite(delta))
        return fail(PD_ERR_ARG, "K and delta must be finite and > 0");
    const double d4 = delta * delta * delta * delta;
    *c_out = 18.0 * K / (M_PI * d4);
    return PD_OK;
}

pd_status pd_critical_stretch(double G_F, double E, double delta, int32_t dim, double* s_c_out)
{
    if (!s_c_out) return fail(PD_ERR_ARG, "s_c_out is NULL");
    if (!(G_F > 0.0) || !(E > 0.0) || !(delta > 0.0) || !std::isfinite(G_F) ||
        !std::isfinite(E) || !std::isfinite(delta))
        return fail(PD_ERR_ARG, "G_F, E and delta must be finite and > 0");
    switch (dim) {
    case PD_DIM_3D: *s_c_out = std::sqrt(5.0 * G_F / (6.0 * E * delta)); break;
    case PD_PLANE_STRESS: *s_c_out = std::sqrt(4.0 * M_PI * G_F / (9.0 * E * delta)); break;
    case PD_PLANE_STRAIN: *s_c_out = std::sqrt(5.0 * M_PI * G_F / (12.0 * E * delta)); break;
    default: return fail(PD_ERR_ARG, "dim must be PD_DIM_3D, PD_PLANE_STRESS or PD_PLANE_STRAIN");
    }
    return PD_OK;
}

pd_status pd_stiffness_factors(int64_t n, const double* coords, const double* volumes,
                               double horizon, const int64_t* fam_off, const int32_t* fam_idx,
                               int32_t flags, double v0, double dx, double* factor)
{
    if (n < 1 || !coords || !volumes || !fam_off || !fam_idx || !factor)
        return fail(PD_ERR_ARG, "need n >= 1 and non-NULL coords, volumes, family and factor");
    if (flags < 1 || flags > (PD_STIFF_CONICAL | PD_STIFF_SURFACE | PD_STIFF_PARTIAL))
        return fail(PD_ERR_ARG,
                    "flags must combine PD_STIFF_CONICAL, PD_STIFF_SURFACE and PD_STIFF_PARTIAL");
    if ((flags & PD_STIFF_PARTIAL) && !(dx > 0.0 && std::isfinite(dx)))
        return fail(PD_ERR_ARG, "the partial volume needs a finite lattice spacing dx > 0");
    if (!(horizon > 0.0) || !std::isfinite(horizon))
        return fail(PD_ERR_ARG, "horizon must be finite and > 0");
    if ((flags & PD_STIFF_SURFACE) && !(v0 > 0.0 && std::isfinite(v0)))
        return fail(PD_ERR_ARG, "the surface correction needs a finite v0 > 0");
    const std::string msg = check_family(n, fam_off, fam_idx);
    if (!msg.empty()) return fail(PD_ERR_ARG, "%s", msg.c_str());
    stiffness_factors(n, coords, volumes, horizon, fam_off, fam_idx, flags, v0, dx, factor);
    return PD_OK;
}

}  // extern "C"

namespace {

pd_status check_cfg(const pd_config* cfg)
{
    if (cfg->precision != PD_PREC_F32 && cfg->precision != PD_PREC_F64 &&
        cfg->precision != PD_PREC_DW)
        return fail(PD_ERR_ARG, "precision must be PD_PREC_F32, PD_PREC_F64 or PD_PREC_DW");
    if (!(cfg->dt > 0.0) || !(cfg->density > 0.0) || !(cfg->damping >= 0.0) ||
        !std::isfinite(cfg->dt) || !std::isfinite(cfg->density) || !std::isfinite(cfg->damping))
        return fail(PD_ERR_ARG, "dt and density must be > 0, damping >= 0");
    if (cfg->graph_steps < 0 || cfg->graph_steps > 4096)
        return fail(PD_ERR_ARG, "graph_steps must be in [0, 4096]");
    if (cfg->block_threads != 0 &&
        (cfg->block_threads < 32 || cfg->block_threads > 256 || cfg->block_threads % 32))
        return fail(PD_ERR_ARG, "block_threads must be a multiple of 32 in [32, 256]");
    if (cfg->reorder != 0 && cfg->reorder != 1) return fail(PD_ERR_ARG, "reorder must be 0 or 1");
    if (cfg->integrator != PD_INTEGRATOR_EC && cfg->integrator != PD_INTEGRATOR_VV)
        return fail(PD_ERR_ARG, "integrator must be PD_INTEGRATOR_EC or PD_INTEGRATOR_VV");
    if (cfg->general != 0 && cfg->general != 1) return fail(PD_ERR_ARG, "general must be 0 or 1");
    if (cfg->lat_variant < 0 || cfg->lat_variant > 1 + kLatTmaShapes)
        return fail(PD_ERR_ARG, "lat_variant must be in [0, %d]", 1 + kLatTmaShapes);
    return PD_OK;
}

pd_status check_material(const pd_material* mat)
{
    if (!(mat->c > 0.0) || !std::isfinite(mat->c)) return fail(PD_ERR_ARG, "c must be > 0");
    if (mat->sc_mode == 0) {
        if (!(mat->sc > 0.0) || !std::isfinite(mat->sc)) return fail(PD_ERR_ARG, "sc must be > 0");
    } else if (mat->sc_mode == 1) {
        if (!(mat->sc_lo > 0.0) || !(mat->sc_hi > mat->sc_lo) || !std::isfinite(mat->sc_hi))
            return fail(PD_ERR_ARG, "need 0 < sc_lo < sc_hi");
    } else {
        return fail(PD_ERR_ARG, "sc_mode must be 0 or 1");
    }
    if (mat->kr != 0.0 && !(mat->kr >= 1.0 && std::isfinite(mat->kr)))
        return fail(PD_ERR_ARG, "kr must be 0 (PMB) or a finite value >= 1 (bilinear softening)");
    if (mat->kink_ratio != 0.0 &&
        !(mat->kr > 1.0 && mat->kink_ratio > 1.0 && mat->kink_ratio < mat->kr &&
          mat->kink_force > 0.0 && mat->kink_force <= 1.0))
        return fail(PD_ERR_ARG, "trilinear softening needs kr > kink_ratio > 1 and kink_force in (0, 1]");
    if (mat->model != 0 && mat->model != 1) return fail(PD_ERR_ARG, "model must be 0 or 1");
    if (mat->model == 1) {
        if (!(mat->bulk_modulus > 0.0) || !(mat->shear_modulus >= 0.0) ||
            !std::isfinite(mat->bulk_modulus) || !std::isfinite(mat->shear_modulus))
            return fail(PD_ERR_ARG, "the state-based model needs bulk_modulus > 0, shear_modulus >= 0");
        if (mat->kr != 0.0)
            return fail(PD_ERR_ARG, "softening is not available with the state-based model");
    }
    return PD_OK;
}

pd_status check_body(int64_t n, const double* coords, const double* volumes, double horizon,
                     const double* cuts, int32_t n_cuts, const pd_bc* bc)
{
    if (n < 1 || n >= (int64_t)1 << 31) return fail(PD_ERR_ARG, "n must be in [1, 2^31)");
    if (!coords || !volumes || !bc) return fail(PD_ERR_ARG, "coords, volumes and bc are required");
    if (!bc->type) return fail(PD_ERR_ARG, "bc->type is required");
    if (n_cuts < 0 || (n_cuts > 0 && !cuts)) return fail(PD_ERR_ARG, "invalid cuts");
    if (!(horizon > 0.0) || !std::isfinite(horizon)) return fail(PD_ERR_ARG, "horizon must be > 0");
    if (!std::isfinite(bc->disp_rate) || !std::isfinite(bc->load))
        return fail(PD_ERR_ARG, "disp_rate and load must be finite");
    if (bc->ramp_steps < 0) return fail(PD_ERR_ARG, "ramp_steps must be >= 0");
    if (!finite_all(coords, 3 * n)) return fail(PD_ERR_ARG, "non-finite coordinates");
    for (int64_t i = 0; i < n; ++i)
        if (!(volumes[i] > 0.0) || !std::isfinite(volumes[i]))
            return fail(PD_ERR_ARG, "volumes must be finite and > 0");
    return PD_OK;
}

// Host description of a model whose family (h->off, h->idx, after the cuts)
// and material scalars are already in the handle.
struct ModelDesc {
    int64_t n = 0;
    const double* coords = nullptr;   // 3n
    const double* wvol = nullptr;     // n: w = c * wvol (batches fold c into wvol)
    const uint8_t* type = nullptr;    // 3n
    const double* disp = nullptr;     // 3n or null
    const double* force = nullptr;    // 3n or null
    const uint8_t* no_fail = nullptr; // n or null
    const double* centre = nullptr;   // 3n per-node origin of the FP32 positions, or null
    double unit = 1.0;                // FP32 length unit (the horizon)
    double horizon = 1.0;             // cell size of the optional node reordering
    int uniform_w = -1;               // batches: 1 if every instance has uniform weights
    std::vector<int32_t> inst, hid;   // batches only
    std::vector<InstParams> itab;
    // batches whose instances are all regular-lattice models: their lattices
    // (first = offset in the concatenation) and the lattice order of each
    std::vector<Lattice> lats;
    std::vector<int32_t> lat_perm;
};

pd_status build_device(pd_handle* h, const ModelDesc& d, const pd_config* cfg)
{
    const int64_t n = d.n;
    int64_t maxfam = 0;
    for (int64_t i = 0; i < n; ++i) maxfam = std::max(maxfam, h->off[i + 1] - h->off[i]);
    if (maxfam > PD_MAX_FAMILY)
        return fail(PD_ERR_FAMILY_TOO_LARGE, "largest family has %lld members (max %d)",
                    (long long)maxfam, PD_MAX_FAMILY);
    h->Q = (int)std::max<int64_t>(1, (maxfam + 31) / 32);
    h->n = n;
    h->n_slices = (n + 31) / 32;
    h->n_pad = 32 * h->n_slices;
    h->n_bonds = h->off[n];
    h->dw = cfg->precision == PD_PREC_DW;
    h->precision = h->dw ? PD_PREC_F64 : cfg->precision;
    h->delta = d.unit;
    h->dt = cfg->dt;
    h->eta = cfg->damping;
    h->rho = cfg->density;
    h->graph_steps = cfg->graph_steps;
    h->integrator = cfg->integrator;
    h->block = cfg->block_threads ? cfg->block_threads : 256;
    h->device = cfg->device;
    h->vol0 = d.wvol[0];
    h->uniform_vol = true;
    for (int64_t i = 1; i < n && h->uniform_vol; ++i) h->uniform_vol = d.wvol[i] == d.wvol[0];
    if (d.uniform_w >= 0) h->uniform_vol = d.uniform_w == 1;

    if (cfg->check_dt) {
        const double dtc = stable_dt(n, d.coords, d.wvol, h->off, h->idx, h->c, h->rho);
        if (h->dt > dtc) return fail(PD_ERR_UNSTABLE_DT, "dt = %g exceeds the stable bound %g", h->dt, dtc);
    }

    std::vector<BcClass> table;
    std::vector<uint8_t> cls;
    std::string msg = bc_classes(n, d.type, d.disp, d.force, d.no_fail, table, cls, h->has_nofail);
    if (!msg.empty()) return fail(PD_ERR_ARG, "%s", msg.c_str());

    // FP32 Euler-Cromer PMB models on a regular lattice (the stencil kernel's
    // case): lattice node order and the stencil-ordered layout
    // (a batch whose instances all are: pd_batch_create found their lattices)
    if (!d.lats.empty()) {
        h->lattice = true;
        h->lats = d.lats;
        h->perm = d.lat_perm;
        h->inv.assign(n, 0);
        for (int64_t p = 0; p < n; ++p) h->inv[h->perm[p]] = (int32_t)p;
        h->lat_of.resize(n);
        for (int64_t p = 0; p < n; ++p) h->lat_of[p] = d.inst[h->perm[p]];
    } else {
        h->lats.assign(1, Lattice{});
        h->lattice = cfg->precision == PD_PREC_F32 && (h->model == 0 || h->model == 1) &&
                     h->kr < 1.0 &&
                     h->integrator == PD_INTEGRATOR_EC && h->ramp_steps == 0 && d.inst.empty() &&
                     cfg->reorder == 0 && cfg->general == 0 && h->uniform_vol &&
                     detect_lattice(n, d.coords, h->off, h->idx, h->lats[0], h->perm, h->inv);
    }
    std::vector<int32_t> nbr, sw;
    std::vector<uint32_t> bits;
    if (h->lattice) {
        h->Q = kStencilSlots / 32;
        build_layout_stencil(n, h->off, h->idx, h->perm, h->inv, h->lats,
                             h->lat_of.empty() ? nullptr : &h->lat_of, nbr, bits, sw, h->cnt);
        // the stencil's reach: |o_x Sx + o_y Sy + o_z| <= 3 Sx + 3 Sy + 3
        h->lat_halo = 0;
        for (const Lattice& L : h->lats)
            h->lat_halo = std::max<int64_t>(h->lat_halo, 3 * L.N[1] * L.N[2] + 3 * L.N[2] + 3);
    } else {
        spatial_order(n, d.coords, d.horizon, cfg->reorder, h->perm, h->inv);
        build_layout(n, h->off, h->idx, h->perm, h->inv, h->Q, nbr, bits, sw, h->cnt);
    }

    // ---- device
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if (cfg->stream) {
        h->stream = (cudaStream_t)cfg->stream;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "stream create");
        h->own_stream = true;
    }
    const int64_t np = h->n_pad;
    const bool f32 = h->precision == 32;
#define ALLOC(ptr, type, count)                                      \
    do {                                                             \
        e = h->alloc((type**)&(ptr), (size_t)(count));               \
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc " #ptr); \
    } while (0)
    if (f32 && h->lattice) {
        // published records with a zero halo: the stencil's wrapped reads stay in bounds
        const int64_t H = h->lat_halo;
        for (int k = 0; k < 2; ++k) {
            ALLOC(h->lat_pub[k], float4, np + 2 * H);
            h->lat_pub[k] += H;
            ALLOC(h->lat_u[k], double, 3 * np);
        }
    }
    if (f32) {
        if (!h->lattice) {
            ALLOC(h->rec32[0], float4, 2 * np);
            ALLOC(h->rec32[1], float4, 2 * np);
            ALLOC(h->lo32, float4, np);
        }
        ALLOC(h->w32, float, np);
        ALLOC(h->v, float, 3 * np);
        ALLOC(h->wsum_inv, float, np);
        ALLOC(h->damage, float, np);
    } else {
        ALLOC(h->rec[0], double, 8 * np);
        ALLOC(h->rec[1], double, 8 * np);
        ALLOC(h->v, double, 3 * np);
        ALLOC(h->wsum_inv, double, np);
        ALLOC(h->damage, double, np);
        if (h->dw) {
            ALLOC(h->recdw[0], float4, 4 * np);
            ALLOC(h->recdw[1], float4, 4 * np);
            ALLOC(h->lendw, float2, nbr.size());
        }
        ALLOC(h->ilen, double, nbr.size());  // also the adjoint's
    }
    if (h->model == 1) {
        if (f32) {
            ALLOC(h->osb32_theta, float, np);
            if (h->lattice) {
                ALLOC(h->osblat_coef, float4, np);
                ALLOC(h->osblat_rec, float4, np + 2 * h->lat_halo);
                h->osblat_rec += h->lat_halo;
                ALLOC(h->osblat_b, float, np + 2 * h->lat_halo);
                h->osblat_b += h->lat_halo;
                ALLOC(h->osblat_exact, uint8_t, h->n_slices);
            } else {
                ALLOC(h->osb32_mvol, float, np);
                ALLOC(h->osb32_ab, float2, np);
            }
        } else if (h->dw) {
            ALLOC(h->osb_mvol, double, np);
            ALLOC(h->osb_theta, double, np);
            ALLOC(h->osbdw_ab, float4, np);
        } else {
            ALLOC(h->osb_len, double, nbr.size());
            ALLOC(h->osb_mvol, double, np);
            ALLOC(h->osb_theta, double, np);
            ALLOC(h->osb_alpha, double, np);
            ALLOC(h->osb_beta, double, np);
        }
    }
    if (h->kr >= 1.0) {  // bilinear softening: every bond starts intact, mu = 1
        if (f32)
            ALLOC(h->integ, float, nbr.size());
        else
            ALLOC(h->integ, double, nbr.size());
        e = launch_fill(h->precision, h->integ, (int64_t)nbr.size(), 1.0, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "initial bond integrity");
    }
    ALLOC(h->nbr, int32_t, nbr.size());
    ALLOC(h->bits, uint32_t, bits.size());
    ALLOC(h->bits0, uint32_t, bits.size());
    ALLOC(h->sw, int32_t, sw.size());
    ALLOC(h->bcc, uint8_t, np);
    ALLOC(h->bct, BcClass, table.size());
    ALLOC(h->gid, int32_t, np);
    ALLOC(h->x64, double, 3 * np);
    ALLOC(h->vol, double, np);
    ALLOC(h->err, int, 2);  // [0] step kernels' flags, [1] input checks
    ALLOC(h->step_ctr, int64_t, 2);  // [0] step counter, [1] step of the last set state
    if (h->integrator == PD_INTEGRATOR_VV) {
        if (f32)
            ALLOC(h->vpeek, float, 3 * np);
        else
            ALLOC(h->vpeek, double, 3 * np);
    }
    ALLOC(h->staging, double, 6 * n);  // u and v halves for host transfers
    if (!d.inst.empty()) {
        ALLOC(h->inst, int32_t, np);
        ALLOC(h->hid, int32_t, np);
        ALLOC(h->itab, InstParams, d.itab.size());
    }
#undef ALLOC

    // node data in the library's order (padding nodes: zero volume, class 0)
    double gctr[3];
    {
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) lo[a] = hi[a] = d.coords[a];
        for (int64_t i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], d.coords[3 * i + a]);
                hi[a] = std::max(hi[a], d.coords[3 * i + a]);
            }
        for (int a = 0; a < 3; ++a) gctr[a] = 0.5 * (lo[a] + hi[a]);
        if (h->dw) {
            // double-word positions start B horizons above zero, B above the
            // largest coordinate difference of any bond: then for every bond
            // x_j / x_i is in [1/2, 2] per component, and the difference of the
            // leading words is exact (Sterbenz)
            double maxd = 0.0;
            const int64_t* off = h->off.data();
            const int32_t* idx = h->idx.data();
#pragma omp parallel for reduction(max : maxd) schedule(static)
            for (int64_t i = 0; i < n; ++i)
                for (int64_t k = off[i]; k < off[i + 1]; ++k)
                    for (int a = 0; a < 3; ++a)
                        maxd = std::max(maxd, std::fabs(d.coords[3 * (int64_t)idx[k] + a] -
                                                        d.coords[3 * i + a]));
            const double B = std::ceil(maxd / d.unit) + 1.0;
            for (int a = 0; a < 3; ++a) h->dw_origin[a] = lo[a] - B * d.unit;
        }
    }
    std::vector<double> xs(3 * np, 0.0), vs(np, 0.0), cs(3 * np, 0.0);
    std::vector<uint8_t> clsp(np, 0);
    std::vector<int32_t> gids(np, 0), insts, hids;
    if (!d.inst.empty()) {
        insts.assign(np, 0);
        hids.assign(np, 0);
    }
    for (int64_t p = 0; p < n; ++p) {
        const int64_t i = h->perm[p];
        for (int a = 0; a < 3; ++a) {
            xs[3 * p + a] = d.coords[3 * i + a];
            cs[3 * p + a] = d.centre ? d.centre[3 * i + a] : gctr[a];
        }
        vs[p] = d.wvol[i];
        clsp[p] = cls[i];
        gids[p] = (int32_t)i;
        if (!d.inst.empty()) {
            insts[p] = d.inst[i];
            hids[p] = d.hid[i];
        }
    }
    auto up = [&](void* dst, const void* src, size_t bytes, const char* what) -> pd_status {
        cudaError_t ee = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream);
        if (ee != cudaSuccess) return cuda_fail(ee, what);
        return PD_OK;
    };
    pd_status st;
    std::vector<float4> r32;
    std::vector<double> r64;
    if (f32 && !h->lattice) {  // (lattice: the state starts at zero, as allocated)
        r32.assign(2 * np, make_float4(0.f, 0.f, 0.f, 0.f));
        for (int64_t p = 0; p < n; ++p)
            r32[2 * p] = make_float4((float)((xs[3 * p] - cs[3 * p]) / d.unit),
                                     (float)((xs[3 * p + 1] - cs[3 * p + 1]) / d.unit),
                                     (float)((xs[3 * p + 2] - cs[3 * p + 2]) / d.unit), 0.0f);
        if ((st = up(h->rec32[0], r32.data(), 32 * np, "upload records")) ||
            (st = up(h->rec32[1], r32.data(), 32 * np, "upload records")))
            return st;
    } else if (!f32) {
        r64.assign(8 * np, 0.0);
        for (int64_t p = 0; p < n; ++p)
            for (int a = 0; a < 3; ++a) r64[8 * p + a] = xs[3 * p + a];
        if ((st = up(h->rec[0], r64.data(), 64 * np, "upload records")) ||
            (st = up(h->rec[1], r64.data(), 64 * np, "upload records")))
            return st;
    }
    if ((st = up(h->nbr, nbr.data(), nbr.size() * 4, "upload family")) ||
        (st = up(h->bits, bits.data(), bits.size() * 4, "upload bond flags")) ||
        (st = up(h->bits0, bits.data(), bits.size() * 4, "upload bond flags")) ||
        (st = up(h->sw, sw.data(), sw.size() * 4, "upload slice widths")) ||
        (st = up(h->bcc, clsp.data(), np, "upload bc classes")) ||
        (st = up(h->bct, table.data(), table.size() * sizeof(BcClass), "upload bc table")) ||
        (st = up(h->gid, gids.data(), 4 * np, "upload ids")) ||
        (st = up(h->x64, xs.data(), 24 * np, "upload coordinates")) ||
        (st = up(h->vol, vs.data(), 8 * np, "upload volumes")))
        return st;
    if (!d.inst.empty()) {
        if ((st = up(h->inst, insts.data(), 4 * np, "upload instance ids")) ||
            (st = up(h->hid, hids.data(), 4 * np, "upload local ids")) ||
            (st = up(h->itab, d.itab.data(), d.itab.size() * sizeof(InstParams),
                     "upload instance table")))
            return st;
    }
    if (!f32) {
        e = launch_inv_len(h->x64, h->nbr, h->sw, n, h->Q, h->ilen, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "bond lengths");
    }
    if (h->dw) {
        e = launch_dw_len(h->x64, h->nbr, n, h->Q, 1.0 / h->delta, h->lendw, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "bond lengths");
    }
    if (h->model == 1 && !f32) {
        e = h->dw ? launch_osb_dw_setup(args_f64(h, 0), osbdw_args(h), h->stream)
                  : launch_osb_setup(args_f64(h, 0), osb_args(h), h->x64, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "state-based set-up");
    }
    if ((st = upload_weights(h)) != PD_OK) return st;
    if (h->model == 1 && f32) {  // needs the node weights (volumes)
        if (h->lattice) {
            // weighted volume m~_i = sum_j |xi~|^2 V_j over the family (lattice: the
            // offsets' q; uniform volumes) and the per-node coefficients
            const double kap = h->lats[0].dx / h->delta;
            std::vector<float4> coef((size_t)np, make_float4(0.f, 0.f, 0.f, 0.f));
            for (int64_t p = 0; p < n; ++p) {
                const int64_t i = h->perm[p];
                double m = 0.0;
                for (int64_t k = h->off[i]; k < h->off[i + 1]; ++k) {
                    const int sl = stencil_slot(h->lats[0], p, h->inv[h->idx[k]]);
                    m += kap * kap * stencil_offset(sl).q * h->vol0;
                }
                if (m > 0.0)
                    coef[p] = make_float4((float)(3.0 / m),
                                          (float)((3.0 * h->osb_K - 5.0 * h->osb_G) / (h->delta * m)),
                                          (float)(15.0 * h->osb_G / (h->delta * m)), 0.f);
            }
            std::vector<float> bco((size_t)np);
            for (int64_t p = 0; p < np; ++p) bco[(size_t)p] = coef[(size_t)p].z;
            e = cudaMemcpyAsync(h->osblat_coef, coef.data(), 16 * (size_t)np,
                                cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(h->osblat_b, bco.data(), 4 * (size_t)np, cudaMemcpyHostToDevice,
                                    h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        } else {
            e = launch_osb32_setup(args_f32(h, 0), osb32_args(h), h->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "state-based set-up");
    }
    if (cfg->lat_variant != 0 && !(h->lattice && h->model == 0))
        return fail(PD_ERR_ARG, "lat_variant applies to bond-based lattice handles "
                                "(pd_info_t.layout PD_LAYOUT_LATTICE)");
    if (cfg->lat_variant >= 2 && h->batch)
        return fail(PD_ERR_ARG, "the tile step (lat_variant 2..4) takes single models");
    h->lat_var = cfg->lat_variant;
    h->blocks_per_sm = cfg->blocks_per_sm;
    if ((st = choose_grid(h, h->blocks_per_sm)) != PD_OK) return st;
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    return PD_OK;
}

void set_material(pd_handle* h, const pd_material* mat, const pd_bc* bc)
{
    h->c = mat->c;
    h->kr = mat->kr;
    h->k1 = mat->kink_ratio;
    h->beta = mat->kink_ratio > 1.0 ? mat->kink_force : 1.0;
    h->model = mat->model;
    h->osb_K = mat->bulk_modulus;
    h->osb_G = mat->shear_modulus;
    h->sc_mode = mat->sc_mode;
    h->sc = mat->sc_mode == 0 ? mat->sc : 0.5 * (mat->sc_lo + mat->sc_hi);
    h->sc_seed = mat->sc_seed;
    h->sc_lo = mat->sc_mode == 1 ? mat->sc_lo : mat->sc;
    h->sc_hi = mat->sc_mode == 1 ? mat->sc_hi : mat->sc;
    h->disp_rate = bc->disp_rate;
    h->load = bc->load;
    h->ramp_steps = bc->ramp_steps;
}

}  // namespace

extern "C" {

pd_status pd_create(int64_t n, const double* coords, const double* volumes, double horizon,
                    const int64_t* fam_off, const int32_t* fam_idx, const double* cuts,
                    int32_t n_cuts, const pd_material* mat, const pd_bc* bc,
                    const pd_config* cfg, pd_handle** out)
{
    NvtxScope nvtx_scope_("pd_create");
    g_err.clear();
    if (!out) return fail(PD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!mat || !cfg) return fail(PD_ERR_ARG, "mat and cfg are required");
    pd_status st;
    if ((st = check_body(n, coords, volumes, horizon, cuts, n_cuts, bc)) != PD_OK) return st;
    if ((st = check_cfg(cfg)) != PD_OK || (st = check_material(mat)) != PD_OK) return st;
    if ((fam_off == nullptr) != (fam_idx == nullptr))
        return fail(PD_ERR_ARG, "fam_off and fam_idx must both be given or both be NULL");

    pd_handle* h = new (std::nothrow) pd_handle();
    if (!h) return fail(PD_ERR_OOM, "host allocation");
    std::string msg;
    if (fam_off) {
        msg = check_family(n, fam_off, fam_idx);
        if (msg.empty()) {
            h->off.assign(fam_off, fam_off + n + 1);
            h->idx.assign(fam_idx, fam_idx + fam_off[n]);
        }
    } else {
        msg = search_family(n, coords, horizon, h->off, h->idx);
    }
    if (!msg.empty()) {
        delete h;
        return fail(PD_ERR_ARG, "%s", msg.c_str());
    }
    apply_cuts(n, coords, cuts, n_cuts, h->off, h->idx);
    set_material(h, mat, bc);
    ModelDesc d;
    d.n = n;
    d.coords = coords;
    d.wvol = volumes;
    d.type = bc->type;
    d.disp = bc->disp;
    d.force = bc->force;
    d.no_fail = bc->no_fail;
    d.unit = horizon;
    d.horizon = horizon;
    if ((st = build_device(h, d, cfg)) != PD_OK) {
        h->release();
        delete h;
        return st;
    }
    h->inst_off = {0, n};
    *out = h;
    return PD_OK;
}

pd_status pd_batch_create(int32_t n_inst, const pd_instance* inst, const pd_config* cfg,
                          pd_handle** out)
{
    NvtxScope nvtx_scope_("pd_batch_create");
    g_err.clear();
    if (!out) return fail(PD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_inst < 1 || !inst || !cfg) return fail(PD_ERR_ARG, "need n_inst >= 1, inst and cfg");
    pd_status st;
    if ((st = check_cfg(cfg)) != PD_OK) return st;
    int64_t n = 0;
    double unit = 0.0;
    bool any_nofail = false;
    for (int32_t b = 0; b < n_inst; ++b) {
        const pd_instance& I = inst[b];
        if ((st = check_body(I.n, I.coords, I.volumes, I.horizon, I.cuts, I.n_cuts, &I.bc)) != PD_OK ||
            (st = check_material(&I.mat)) != PD_OK)
            return fail(st, "instance %d: %s", b, g_err.c_str());
        if (I.bc.disp_rate != inst[0].bc.disp_rate || I.bc.load != inst[0].bc.load ||
            I.bc.ramp_steps != inst[0].bc.ramp_steps)
            return fail(PD_ERR_ARG,
                        "instance %d: disp_rate, load and ramp_steps must equal instance 0's", b);
        if (I.mat.model != inst[0].mat.model ||
            (I.mat.model == 1 && (I.mat.bulk_modulus != inst[0].mat.bulk_modulus ||
                                  I.mat.shear_modulus != inst[0].mat.shear_modulus)))
            return fail(PD_ERR_ARG,
                        "instance %d: model, bulk_modulus and shear_modulus must equal instance 0's",
                        b);
        if (I.mat.kr != inst[0].mat.kr || I.mat.kink_ratio != inst[0].mat.kink_ratio ||
            I.mat.kink_force != inst[0].mat.kink_force)
            return fail(PD_ERR_ARG,
                        "instance %d: kr, kink_ratio and kink_force must equal instance 0's", b);
        n += I.n;
        unit = std::max(unit, I.horizon);
        any_nofail = any_nofail || I.bc.no_fail != nullptr;
    }
    if (n >= (int64_t)1 << 31) return fail(PD_ERR_ARG, "batch has 2^31 nodes or more");

    pd_handle* h = new (std::nothrow) pd_handle();
    if (!h) return fail(PD_ERR_OOM, "host allocation");
    std::vector<double> x(3 * n), wv(n), disp(3 * n, 0.0), force(3 * n, 0.0), centre(3 * n);
    std::vector<uint8_t> type(3 * n), nofail(any_nofail ? n : 0, 0);
    ModelDesc d;
    d.inst.resize(n);
    d.hid.resize(n);
    d.itab.resize(n_inst);
    h->off.assign(1, 0);
    h->inst_off.assign(1, 0);
    bool uniform_all = true;  // every instance has uniform volumes
    // FP32 Euler-Cromer PMB batches whose instances all are regular lattices run
    // the stencil kernel, each instance in its own lattice units
    bool all_lattice = cfg->precision == PD_PREC_F32 && inst[0].mat.model == 0 &&
                       inst[0].mat.kr < 1.0 && cfg->integrator == PD_INTEGRATOR_EC &&
                       inst[0].bc.ramp_steps == 0 && cfg->reorder == 0 && cfg->general == 0;
    std::vector<Lattice> lats;
    std::vector<int32_t> lat_perm;
    for (int32_t b = 0; b < n_inst; ++b) {
        const pd_instance& I = inst[b];
        const int64_t o = h->inst_off.back();
        std::vector<int64_t> off;
        std::vector<int32_t> idx;
        std::string msg = search_family(I.n, I.coords, I.horizon, off, idx);
        if (!msg.empty()) {
            delete h;
            return fail(PD_ERR_ARG, "instance %d: %s", b, msg.c_str());
        }
        apply_cuts(I.n, I.coords, I.cuts, I.n_cuts, off, idx);
        if (all_lattice) {
            Lattice L;
            std::vector<int32_t> pb, ib;
            all_lattice = detect_lattice(I.n, I.coords, off, idx, L, pb, ib);
            if (all_lattice) {
                L.first = o;
                lats.push_back(L);
                for (int32_t q : pb) lat_perm.push_back((int32_t)(q + o));
            }
        }
        if (cfg->check_dt && I.mat.model == 1) {
            // the state-based weights are plain volumes: bound each instance with
            // its own PMB-equivalent micromodulus, as for a single model
            const double dtc = stable_dt(I.n, I.coords, I.volumes, off, idx, I.mat.c, cfg->density);
            if (cfg->dt > dtc) {
                delete h;
                return fail(PD_ERR_UNSTABLE_DT, "instance %d: dt = %g exceeds the stable bound %g",
                            b, cfg->dt, dtc);
            }
        }
        for (int64_t i = 0; i < I.n; ++i) h->off.push_back(h->off.back() + (off[i + 1] - off[i]));
        for (int32_t j : idx) h->idx.push_back((int32_t)(j + o));
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) lo[a] = hi[a] = I.coords[a];
        for (int64_t i = 0; i < I.n; ++i)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], I.coords[3 * i + a]);
                hi[a] = std::max(hi[a], I.coords[3 * i + a]);
            }
        for (int64_t i = 0; i < I.n; ++i) {
            const int64_t k = o + i;
            for (int a = 0; a < 3; ++a) {
                x[3 * k + a] = I.coords[3 * i + a];
                centre[3 * k + a] = 0.5 * (lo[a] + hi[a]);
                type[3 * k + a] = I.bc.type[3 * i + a];
                if (I.bc.disp) disp[3 * k + a] = I.bc.disp[3 * i + a];
                if (I.bc.force) force[3 * k + a] = I.bc.force[3 * i + a];
            }
            // bond-based weights carry the instance's micromodulus; the state-based
            // model's are the volumes
            wv[k] = (I.mat.model == 1 ? 1.0 : I.mat.c) * I.volumes[i];
            if (I.bc.no_fail) nofail[k] = I.bc.no_fail[i];
            d.inst[k] = b;
            d.hid[k] = (int32_t)i;
        }
        InstParams& ip = d.itab[b];
        ip.sc_mode = I.mat.sc_mode;
        ip.sc = I.mat.sc_mode == 0 ? I.mat.sc : 0.5 * (I.mat.sc_lo + I.mat.sc_hi);
        ip.sc_lo = I.mat.sc_mode == 1 ? I.mat.sc_lo : I.mat.sc;
        ip.sc_hi = I.mat.sc_mode == 1 ? I.mat.sc_hi : I.mat.sc;
        ip.sc_seed = I.mat.sc_seed;
        // softening: the band below the smallest s_0 = s_c / kr is resolved too
        ip.fast_lo = (float)((1.0 - 2.0 * kGuard) * ip.sc_lo /
                             (inst[0].mat.kr >= 1.0 ? inst[0].mat.kr : 1.0));
        ip.w_const = (float)((I.mat.model == 1 ? 1.0 : I.mat.c) * I.volumes[0]);
        if (all_lattice) {
            const Lattice& L = lats.back();
            const double f = (1.0 - 2.0 * kGuard) * ip.sc_lo;
            ip.lat_sx = (int32_t)(L.N[1] * L.N[2]);
            ip.lat_sy = (int32_t)L.N[2];
            ip.lat_thr_t = (float)(f * (2.0 + f));
            const double tu = std::min(f * (2.0 + f), kLatPolyX);  // per unit q (kappa = 1)
            ip.lat_cc_t = (float)(0.5 * (tu - kLatPolyX));
            ip.lat_ch_t = (float)(0.5 * (tu + kLatPolyX));
            ip.dtd = (float)(cfg->dt / L.dx);
            ip.unit = L.dx;
            ip.inv_unit = 1.0 / L.dx;
        }
        for (int64_t i = 1; i < I.n && uniform_all; ++i) uniform_all = I.volumes[i] == I.volumes[0];
        h->inst_off.push_back(o + I.n);
    }
    // weights carry each instance's micromodulus: w = 1 * (c_b V)
    pd_material m0 = inst[0].mat;
    m0.c = 1.0;
    set_material(h, &m0, &inst[0].bc);
    h->batch = true;
    d.n = n;
    d.coords = x.data();
    d.wvol = wv.data();
    d.type = type.data();
    d.disp = disp.data();
    d.force = force.data();
    d.no_fail = any_nofail ? nofail.data() : nullptr;
    d.centre = centre.data();
    d.unit = unit;
    d.horizon = unit;
    d.uniform_w = uniform_all ? 1 : 0;
    if (all_lattice && uniform_all) {
        d.lats = lats;
        d.lat_perm = lat_perm;
    }
    if ((st = build_device(h, d, cfg)) != PD_OK) {
        h->release();
        delete h;
        return st;
    }
    *out = h;
    return PD_OK;
}

pd_status pd_batch_offsets(pd_handle* h, int32_t* n_inst, int64_t* node_offset)
{
    if (!h) return fail(PD_ERR_ARG, "NULL handle");
    const int32_t k = (int32_t)h->inst_off.size() - 1;
    if (n_inst) *n_inst = k;
    if (node_offset) std::memcpy(node_offset, h->inst_off.data(), sizeof(int64_t) * (k + 1));
    return PD_OK;
}

}  // extern "C"

extern "C" {

void pd_destroy(pd_handle* h)
{
    if (!h) return;
    h->release();
    delete h;
}

pd_status pd_get_info(pd_handle* h, pd_info_t* out)
{
    if (!h || !out) return fail(PD_ERR_ARG, "NULL argument");
    out->n = h->n;
    out->n_bonds = h->n_bonds;
    out->step = h->step;
    out->precision = h->dw ? PD_PREC_DW : h->precision;
    out->ell_width = 32 * h->Q;
    out->device_bytes = h->device_bytes;
    out->layout = h->lattice ? PD_LAYOUT_LATTICE : PD_LAYOUT_SELL;
    out->lat_variant = h->lattice ? h->lat_var : 0;
    out->step_registers = 0;
    cudaFuncAttributes fa;
    if (cudaSetDevice(h->device) == cudaSuccess &&
        cudaFuncGetAttributes(&fa, step_kernel_fn(h)) == cudaSuccess)
        out->step_registers = fa.numRegs;
    else
        cudaGetLastError();
    return PD_OK;
}

pd_status pd_get_family(pd_handle* h, int64_t* off, int32_t* idx)
{
    if (!h || !off) return fail(PD_ERR_ARG, "NULL argument");
    std::memcpy(off, h->off.data(), sizeof(int64_t) * (h->n + 1));
    if (idx) std::memcpy(idx, h->idx.data(), sizeof(int32_t) * h->n_bonds);
    return PD_OK;
}

pd_status pd_step(pd_handle* h, int64_t n_steps)
{
    NvtxScope nvtx_scope_("pd_step");
    if (!h) return fail(PD_ERR_ARG, "NULL handle");
    if (n_steps < 0) return fail(PD_ERR_ARG, "n_steps must be >= 0");
    if (n_steps == 0) return PD_OK;
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    int64_t left = n_steps;
    const int G = h->graph_steps;
    if (G > 0 && left >= G) {
        if (!h->graph) {
            cudaGraph_t g = nullptr;
            PD_CUDA(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal),
                    "begin capture");
            cudaError_t e = cudaSuccess;
            for (int k = 0; k < G && e == cudaSuccess; ++k) e = launch_one(h, k);
            if (e == cudaSuccess) e = launch_advance(h->step_ctr, G, h->stream);
            cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
            if (e != cudaSuccess || e2 != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return cuda_fail(e != cudaSuccess ? e : e2, "graph capture");
            }
            e = cudaGraphInstantiate(&h->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                h->graph = nullptr;
                return cuda_fail(e, "graph instantiate");
            }
        }
        while (left >= G) {
            PD_CUDA(cudaGraphLaunch(h->graph, h->stream), "graph launch");
            left -= G;
            h->step += G;
        }
    }
    // direct launches: the FP32 lattice kernels take their absolute step and
    // advance the device counter themselves (one launch per step); the others
    // read counter + k and one advance follows
    const bool self_adv = h->lattice && h->precision == 32;
    for (int64_t k = 0; k < left; ++k)
        PD_CUDA(self_adv ? launch_one(h, 0, h->step + k) : launch_one(h, (int)k), "step launch");
    if (left > 0) {
        if (!self_adv) PD_CUDA(launch_advance(h->step_ctr, left, h->stream), "advance");
        h->step += left;
    }
    h->damage_fresh = true;
    return PD_OK;
}

pd_status pd_sync(pd_handle* h)
{
    if (!h) return fail(PD_ERR_ARG, "NULL handle");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    return check_dev_err(h);
}

pd_status pd_get_state(pd_handle* h, double* u, double* v, int64_t* step)
{
    NvtxScope nvtx_scope_("pd_get_state");
    if (!h) return fail(PD_ERR_ARG, "NULL handle");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    const int cur = (int)(h->step & 1);
    const void* vsrc = h->v;
    if (v && h->integrator == PD_INTEGRATOR_VV) {
        pd_status st = vv_force_pass(h);
        if (st != PD_OK) return st;
        vsrc = h->vpeek;
    }
    double* outs[2] = {u, v};
    for (int w = 0; w < 2; ++w) {
        double* o = outs[w];
        if (!o) continue;
        const bool dev = is_device_ptr(o);
        double* dst = dev ? o : h->staging;
        double* uo = w == 0 ? dst : nullptr;
        double* vo = w == 1 ? dst : nullptr;
        if (h->lattice)
            PD_CUDA(launch_get_state_lat(h->lat_u[cur], (const float*)vsrc, h->gid, h->n,
                                         h->delta, h->batch ? h->inst : nullptr, h->itab, uo,
                                         vo, h->stream),
                    "get state");
        else if (h->precision == 32)
            PD_CUDA(launch_get_state_f32(h->rec32[cur], h->lo32, (const float*)vsrc, h->gid,
                                         h->n, h->delta, uo, vo, h->stream),
                    "get state");
        else
            PD_CUDA(launch_get_state_f64(h->rec[cur], (const double*)vsrc, h->gid, h->n, uo, vo,
                                         h->stream),
                    "get state");
        if (!dev)
            PD_CUDA(cudaMemcpyAsync(o, h->staging, 24 * h->n, cudaMemcpyDeviceToHost, h->stream),
                    "copy state to host");
    }
    if (step) *step = h->step;
    return check_dev_err(h);
}

pd_status pd_set_state(pd_handle* h, const double* u, const double* v, int64_t step)
{
    NvtxScope nvtx_scope_("pd_set_state");
    if (!h) return fail(PD_ERR_ARG, "NULL handle");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    // stage host inputs (u and v halves of the staging area), check their values
    // on the device (device inputs are the caller's responsibility, as before),
    // and only then change the state
    const double* ins[2] = {u, v};
    const double* src[2] = {nullptr, nullptr};
    int* chk = h->err + 1;
    PD_CUDA(cudaMemsetAsync(chk, 0, sizeof(int), h->stream), "clear input flag");
    for (int w = 0; w < 2; ++w) {
        if (!ins[w]) continue;
        src[w] = ins[w];
        if (!is_device_ptr(ins[w])) {
            double* dst = h->staging + 3 * h->n * w;
            PD_CUDA(cudaMemcpyAsync(dst, ins[w], 24 * h->n, cudaMemcpyHostToDevice, h->stream),
                    "copy state to device");
            src[w] = dst;
            PD_CUDA(launch_check_finite(src[w], 3 * h->n, chk, h->stream), "check state");
        }
    }
    int bad = 0;
    PD_CUDA(cudaMemcpyAsync(&bad, chk, sizeof(int), cudaMemcpyDeviceToHost, h->stream),
            "read input flag");
    PD_CUDA(cudaStreamSynchronize(h->stream), "synchronize");
    if (bad) return fail(PD_ERR_ARG, "non-finite state");
    if (step >= 0 && step != h->step) {
        h->step = step;
        PD_CUDA(cudaMemcpyAsync(h->step_ctr, &h->step, sizeof(int64_t), cudaMemcpyHostToDevice,
                                h->stream),
                "set step");
    }
    const int cur = (int)(h->step & 1);
    if (src[0] || src[1]) {
        if (h->lattice)
            PD_CUDA(launch_set_state_lat(src[0], src[1], h->gid, h->n, 1.0 / h->delta,
                                         h->batch ? h->inst : nullptr, h->itab, h->lat_u[cur],
                                         h->lat_pub[cur], (float*)h->v, h->stream),
                    "set state");
        else if (h->precision == 32)
            PD_CUDA(launch_set_state_f32(src[0], src[1], h->gid, h->n, 1.0 / h->delta,
                                         h->rec32[cur], h->lo32, (float*)h->v, h->stream),
                    "set state");
        else
            PD_CUDA(launch_set_state_f64(src[0], src[1], h->gid, h->n, h->rec[cur],
                                         (double*)h->v, h->stream),
                    "set state");
        if (h->dw)
            PD_CUDA(launch_dw_publish(h->rec[cur], h->recdw[cur], h->n_pad, h->dw_origin,
                                      1.0 / h->delta, h->stream),
                    "double-word records");
    }
    // the velocity-Verlet history starts again at this step (a^n formed afresh);
    // the host inputs were consumed before the check above, so nothing more
    // needs to finish before returning
    PD_CUDA(cudaMemcpyAsync(h->step_ctr + 1, &h->step, sizeof(int64_t), cudaMemcpyHostToDevice,
                            h->stream),
            "set history start");
    h->vv_start = h->step;
    PD_CUDA(cudaMemsetAsync(h->err, 0, sizeof(int), h->stream), "clear error flag");
    h->damage_fresh = false;
    h->peek_step = -1;
    return PD_OK;
}

pd_status pd_get_bonds(pd_handle* h, uint8_t* mu)
{
    NvtxScope nvtx_scope_("pd_get_bonds");
    if (!h || !mu) return fail(PD_ERR_ARG, "NULL argument");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    pd_status st = vv_force_pass(h);
    if (st != PD_OK) return st;
    std::vector<int64_t> pos;
    st = canonical_slots(h, pos);
    if (st != PD_OK) return st;
    std::vector<uint32_t> bits((size_t)(h->n_slices * h->Q * 32));
    PD_CUDA(cudaMemcpy(bits.data(), h->bits, bits.size() * 4, cudaMemcpyDeviceToHost),
            "copy bond flags");
    const int64_t W = 32LL * h->Q;
    for (int64_t p = 0; p < h->n; ++p) {
        const int64_t g = p / 32, l = p % 32;
        for (int64_t m = 0; m < W; ++m) {
            const int64_t k = pos[(g * W + m) * 32 + l];
            if (k >= 0) mu[k] = (bits[(g * h->Q + (m >> 5)) * 32 + l] >> (m & 31)) & 1u;
        }
    }
    return PD_OK;
}

pd_status pd_get_bond_integrity(pd_handle* h, double* mu)
{
    if (!h || !mu) return fail(PD_ERR_ARG, "NULL argument");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    pd_status st = vv_force_pass(h);
    if (st != PD_OK) return st;
    std::vector<int64_t> pos;
    if ((st = canonical_slots(h, pos)) != PD_OK) return st;
    const int64_t W = 32LL * h->Q;
    std::vector<uint32_t> bits((size_t)(h->n_slices * h->Q * 32));
    PD_CUDA(cudaMemcpy(bits.data(), h->bits, bits.size() * 4, cudaMemcpyDeviceToHost),
            "copy bond flags");
    const size_t ns = (size_t)(h->n_slices * 32 * W);
    std::vector<double> m64;
    std::vector<float> m32;
    if (h->integ) {
        if (h->precision == 32) {
            m32.resize(ns);
            PD_CUDA(cudaMemcpy(m32.data(), h->integ, ns * 4, cudaMemcpyDeviceToHost), "copy integrity");
        } else {
            m64.resize(ns);
            PD_CUDA(cudaMemcpy(m64.data(), h->integ, ns * 8, cudaMemcpyDeviceToHost), "copy integrity");
        }
    }
    for (int64_t p = 0; p < h->n; ++p) {
        const int64_t g = p / 32, l = p % 32;
        for (int64_t m = 0; m < W; ++m) {
            const int64_t slot = (g * W + m) * 32 + l;
            if (pos[(size_t)slot] < 0) continue;
            const bool intact = (bits[(g * h->Q + (m >> 5)) * 32 + l] >> (m & 31)) & 1u;
            double v = intact ? 1.0 : 0.0;
            if (intact && h->integ)
                v = h->precision == 32 ? (double)m32[(size_t)slot] : m64[(size_t)slot];
            mu[pos[(size_t)slot]] = v;
        }
    }
    return PD_OK;
}

pd_status pd_set_bonds(pd_handle* h, const uint8_t* mu)
{
    NvtxScope nvtx_scope_("pd_set_bonds");
    if (!h || !mu) return fail(PD_ERR_ARG, "NULL argument");
    for (int64_t k = 0; k < h->n_bonds; ++k)
        if (mu[k] > 1) return fail(PD_ERR_ARG, "bond flags must be 0 or 1");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    std::vector<int64_t> pos;
    pd_status st = canonical_slots(h, pos);
    if (st != PD_OK) return st;
    const int64_t W = 32LL * h->Q;
    std::vector<uint32_t> bits((size_t)(h->n_slices * h->Q * 32), 0u);
    for (int64_t p = 0; p < h->n; ++p) {
        const int64_t g = p / 32, l = p % 32;
        for (int64_t m = 0; m < W; ++m) {
            const int64_t k = pos[(g * W + m) * 32 + l];
            if (k >= 0 && mu[k]) bits[(g * h->Q + (m >> 5)) * 32 + l] |= 1u << (m & 31);
        }
    }
    PD_CUDA(cudaMemcpyAsync(h->bits, bits.data(), bits.size() * 4, cudaMemcpyHostToDevice, h->stream),
            "upload bond flags");
    if (h->integ) {  // a fresh bond state: intact bonds unsoftened, broken ones 0
        const size_t ns = (size_t)(h->n_slices * 32 * W);
        std::vector<double> m64;
        std::vector<float> m32;
        if (h->precision == 32) m32.assign(ns, 0.0f); else m64.assign(ns, 0.0);
        for (int64_t p = 0; p < h->n; ++p) {
            const int64_t g = p / 32, l = p % 32;
            for (int64_t m = 0; m < W; ++m)
                if ((bits[(g * h->Q + (m >> 5)) * 32 + l] >> (m & 31)) & 1u) {
                    const size_t slot = (size_t)((g * W + m) * 32 + l);
                    if (h->precision == 32) m32[slot] = 1.0f; else m64[slot] = 1.0;
                }
        }
        if (h->precision == 32)
            PD_CUDA(cudaMemcpyAsync(h->integ, m32.data(), ns * 4, cudaMemcpyHostToDevice, h->stream), "upload integrity");
        else
            PD_CUDA(cudaMemcpyAsync(h->integ, m64.data(), ns * 8, cudaMemcpyHostToDevice, h->stream), "upload integrity");
    }
    h->damage_fresh = false;
    h->peek_step = -1;
    return PD_OK;
}

pd_status pd_remove_bonds(pd_handle* h, const int64_t* pairs, int64_t m)
{
    NvtxScope nvtx_scope_("pd_remove_bonds");
    if (!h || (m > 0 && !pairs) || m < 0) return fail(PD_ERR_ARG, "need a handle, m >= 0 and pairs");
    if (m == 0) return PD_OK;
    // every pair is checked before anything changes.  The slot of a directed
    // bond a -> b: the layout lists node a's family in ascending device
    // position, so it is the rank of inv[b] in that row.
    const int64_t W = 32LL * h->Q;
    std::vector<int64_t> word, slot;
    std::vector<uint32_t> mask;
    word.reserve((size_t)(2 * m));
    slot.reserve((size_t)(2 * m));
    mask.reserve((size_t)(2 * m));
    for (int64_t e = 0; e < m; ++e) {
        const int64_t i = pairs[2 * e], j = pairs[2 * e + 1];
        if (i < 0 || j < 0 || i >= h->n || j >= h->n || i == j)
            return fail(PD_ERR_ARG, "pair %lld: (%lld, %lld) is not a pair of distinct nodes",
                        (long long)e, (long long)i, (long long)j);
        for (int dir = 0; dir < 2; ++dir) {
            const int64_t a = dir ? j : i, b = dir ? i : j;
            const int32_t* lo = h->idx.data() + h->off[a];
            const int32_t* hi = h->idx.data() + h->off[a + 1];
            const int32_t* it = std::lower_bound(lo, hi, (int32_t)b);  // rows are sorted
            if (it == hi || *it != b)
                return fail(PD_ERR_ARG, "pair %lld: %lld -> %lld is not a bond of the family",
                            (long long)e, (long long)a, (long long)b);
            const int32_t pb = h->inv[(size_t)b];
            int64_t mm = 0;
            if (h->lattice) {  // stencil-ordered layout: the slot of the lattice offset
                const int64_t pa = h->inv[(size_t)a];
                mm = stencil_slot(h->lats[h->lat_of.empty() ? 0 : h->lat_of[(size_t)pa]], pa, pb);
            } else {
                for (const int32_t* q = lo; q < hi; ++q) mm += h->inv[(size_t)*q] < pb ? 1 : 0;
            }
            const int64_t p = h->inv[(size_t)a], g = p / 32, l = p % 32;
            word.push_back((g * h->Q + (mm >> 5)) * 32 + l);
            mask.push_back(1u << (mm & 31));
            slot.push_back((g * W + mm) * 32 + l);
        }
    }
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    pd_status st = vv_force_pass(h);  // a pending Velocity-Verlet force pass sees the old bonds
    if (st != PD_OK) return st;
    const size_t nk = word.size();
    int64_t* d_word = nullptr;
    int64_t* d_slot = nullptr;
    uint32_t* d_mask = nullptr;
    cudaError_t e = cudaMalloc(&d_word, nk * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_slot, nk * 8);
    if (e == cudaSuccess) e = cudaMalloc(&d_mask, nk * 4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_word, word.data(), nk * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_slot, slot.data(), nk * 8, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_mask, mask.data(), nk * 4, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = launch_clear_slots(h->bits, d_word, d_mask, d_slot, (int64_t)nk, h->precision,
                               h->integ, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(d_word);
    cudaFree(d_slot);
    cudaFree(d_mask);
    PD_CUDA(e, "remove bonds");
    h->damage_fresh = false;
    h->peek_step = -1;
    return PD_OK;
}

pd_status pd_damage(pd_handle* h, double* phi)
{
    NvtxScope nvtx_scope_("pd_damage");
    if (!h || !phi) return fail(PD_ERR_ARG, "NULL argument");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    pd_status st = vv_force_pass(h);
    if (st != PD_OK) return st;
    const bool dev = is_device_ptr(phi);
    double* dst = dev ? phi : h->staging;
    if (h->damage_fresh)  // written by the last step kernel (fused)
        PD_CUDA(launch_gather_damage(h->precision, h->damage, h->gid, h->n, dst, h->stream),
                "damage");
    else
        PD_CUDA(launch_damage(h->precision, h->wrec(), h->nbr, h->bits, h->sw, h->wsum_inv,
                              h->gid, h->n, h->Q, h->integ, dst, h->stream),
                "damage");
    if (!dev)
        PD_CUDA(cudaMemcpyAsync(phi, h->staging, 8 * h->n, cudaMemcpyDeviceToHost, h->stream),
                "copy damage");
    return check_dev_err(h);
}

pd_status pd_adjoint_forward(pd_handle* h, int64_t n_steps, int64_t checkpoint_every)
{
    NvtxScope nvtx_scope_("pd_adjoint_forward");
    if (!h) return fail(PD_ERR_ARG, "NULL handle");
    if (h->precision != 64 || h->batch || h->integ || h->model != 0)
        return fail(PD_ERR_STATE,
                    "the adjoint is available on FP64 and PD_PREC_DW single-model PMB handles");
    if (n_steps < 1 || checkpoint_every < 0)
        return fail(PD_ERR_ARG, "need n_steps >= 1 and checkpoint_every >= 0");
    const bool vv = h->integrator == PD_INTEGRATOR_VV;
    if (vv && h->vv_start != h->step)
        return fail(PD_ERR_STATE,
                    "a velocity-Verlet adjoint run starts from a state set by pd_set_state "
                    "(or at creation), where the acceleration is formed afresh");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    auto& T = h->tape;
    int64_t C = checkpoint_every > 0 ? std::min(checkpoint_every, n_steps)
                                     : (int64_t)std::ceil(std::sqrt((double)n_steps));
    C = std::max<int64_t>(1, C);
    const int64_t nck = (n_steps + C - 1) / C;
    const int64_t np3 = 3 * h->n_pad;
    cudaError_t e;
    if (T.cap_ck < nck) {
        if ((e = h->alloc(&T.ck_u, (size_t)(nck * np3))) != cudaSuccess ||
            (e = h->alloc(&T.ck_v, (size_t)(nck * np3))) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc checkpoints");
        T.cap_ck = nck;
    }
    if (T.cap_seg < C) {
        if ((e = h->alloc(&T.seg, (size_t)(C * np3))) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc segment");
        T.cap_seg = C;
    }
    if (!T.fin_u) {
        if ((e = h->alloc(&T.fin_u, (size_t)np3)) != cudaSuccess ||
            (e = h->alloc(&T.fin_v, (size_t)np3)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc final state");
    }
    T.valid = false;
    h->frozen = true;
    h->drop_graph();
    const int64_t step0 = h->step;
    for (int64_t k = 0; k < n_steps; k += C) {
        const int cur = (int)(h->step & 1);
        PD_CUDA(launch_extract_u(h->rec[cur], h->n_pad, T.ck_u + (k / C) * np3, h->stream),
                "checkpoint u");
        PD_CUDA(cudaMemcpyAsync(T.ck_v + (k / C) * np3, h->v, 8 * np3, cudaMemcpyDeviceToDevice,
                                h->stream),
                "checkpoint v");
        pd_status st = pd_step(h, std::min(C, n_steps - k));
        if (st != PD_OK) {
            h->frozen = false;
            h->drop_graph();
            return st;
        }
    }
    const int cur = (int)(h->step & 1);
    PD_CUDA(launch_extract_u(h->rec[cur], h->n_pad, T.fin_u, h->stream), "final u");
    PD_CUDA(cudaMemcpyAsync(T.fin_v, h->v, 8 * np3, cudaMemcpyDeviceToDevice, h->stream),
            "final v");
    h->frozen = false;
    h->drop_graph();
    T.N = n_steps;
    T.C = C;
    T.nck = nck;
    T.step0 = step0;
    T.vv = vv;
    T.valid = true;
    return check_dev_err(h);
}

pd_status pd_adjoint_backward(pd_handle* h, const double* dLdu, const double* dLdv,
                              double* dL_dc, double* dL_dload, double* dL_du0, double* dL_dv0)
{
    NvtxScope nvtx_scope_("pd_adjoint_backward");
    if (!h) return fail(PD_ERR_ARG, "NULL handle");
    auto& T = h->tape;
    if (!T.valid) return fail(PD_ERR_STATE, "no recorded adjoint forward run");
    if (!dLdu) return fail(PD_ERR_ARG, "dLdu is required");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    const int64_t np3 = 3 * h->n_pad;
    const int64_t slots = h->n_slices * 32LL * h->Q * 32;
    cudaError_t e;
    if (!T.w) {
        if ((e = h->alloc(&T.ub[0], (size_t)np3)) != cudaSuccess ||
            (e = h->alloc(&T.ub[1], (size_t)np3)) != cudaSuccess ||
            (e = h->alloc(&T.vb[0], (size_t)np3)) != cudaSuccess ||
            (e = h->alloc(&T.vb[1], (size_t)np3)) != cudaSuccess ||
            (e = h->alloc(&T.ubm, (size_t)np3)) != cudaSuccess ||
            (e = h->alloc(&T.w, (size_t)np3)) != cudaSuccess ||
            (e = h->alloc(&T.gc, (size_t)slots)) != cudaSuccess ||
            (e = h->alloc(&T.gl, (size_t)h->n_pad)) != cudaSuccess ||
            (e = h->alloc(&T.out, 1)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc adjoint buffers");
        T.n_partial = sum_partials_needed(h->n);
        if ((e = h->alloc(&T.partial, (size_t)T.n_partial)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc reduction scratch");
    }
    if (h->dw && !T.gcdw) {
        if ((e = h->alloc(&T.rrec, (size_t)(4 * h->n_pad))) != cudaSuccess ||
            (e = h->alloc(&T.wrec, (size_t)(2 * h->n_pad))) != cudaSuccess ||
            (e = h->alloc(&T.gcdw, (size_t)slots)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc double-word adjoint buffers");
    }
    // seed: dL/du^N, dL/dv^N in library order
    auto to_lib = [&](const double* src, double* dst) -> pd_status {
        if (!src) {
            PD_CUDA(cudaMemsetAsync(dst, 0, 8 * np3, h->stream), "memset");
            return PD_OK;
        }
        const double* s = src;
        if (!is_device_ptr(src)) {
            PD_CUDA(cudaMemcpyAsync(h->staging, src, 24 * h->n, cudaMemcpyHostToDevice, h->stream),
                    "copy gradient to device");
            s = h->staging;
        }
        PD_CUDA(launch_to_lib3(s, h->gid, h->n, dst, h->stream), "reorder");
        PD_CUDA(cudaStreamSynchronize(h->stream), "synchronize");
        return PD_OK;
    };
    pd_status st;
    PD_CUDA(cudaMemsetAsync(T.ub[0], 0, 8 * np3, h->stream), "memset");
    PD_CUDA(cudaMemsetAsync(T.vb[0], 0, 8 * np3, h->stream), "memset");
    if ((st = to_lib(dLdu, T.ub[0])) != PD_OK || (st = to_lib(dLdv, T.vb[0])) != PD_OK) return st;
    PD_CUDA(cudaMemsetAsync(T.gc, 0, 8 * slots, h->stream), "memset");
    PD_CUDA(cudaMemsetAsync(T.gl, 0, 8 * h->n_pad, h->stream), "memset");
    if (h->dw) PD_CUDA(cudaMemsetAsync(T.gcdw, 0, 8 * slots, h->stream), "memset");

    int sms = 0;
    PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device), "sm count");
    const int agrid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8,
                                                                  (h->n_slices + 7) / 8));
    AdjArgs A{};
    A.x64 = h->x64;
    A.nbr = h->nbr;
    A.bits = h->bits;
    A.sw = h->sw;
    A.Q = h->Q;
    A.vol = h->vol;
    A.cbond = h->per_bond_c ? (const double*)h->cbond : nullptr;
    A.ilen = h->ilen;
    A.c = h->c;
    A.gc = T.gc;
    A.gl = T.gl;
    A.bcc = h->bcc;
    A.bct = h->bct;
    A.dt_rho = h->dt / h->rho;
    A.damp = 1.0 - h->dt * h->eta / h->rho;
    A.n = h->n;
    AdjDwArgs D{};
    if (h->dw) {
        D.rec = T.rrec;
        D.wrec = T.wrec;
        D.len = h->lendw;
        D.cb = h->per_bond_c ? h->cbdw : nullptr;
        const float ch = (float)h->c;
        D.c = make_float2(ch, (float)(h->c - (double)ch));
        D.gc = T.gcdw;
        D.w = T.w;
        D.ubm = T.ubm;
        D.gl = T.gl;
        D.nbr = h->nbr;
        D.bits = h->bits;
        D.sw = h->sw;
        D.Q = h->Q;
        D.uniform_w = h->uniform_vol ? 1 : 0;
        D.n = h->n;
        D.bcc = h->bcc;
        D.bct = h->bct;
        D.dt_rho = A.dt_rho;
        D.damp = A.damp;
        D.inv_delta = 1.0 / h->delta;
        D.vol0 = h->vol0;
    }

    h->frozen = true;
    h->drop_graph();
    int cb = 0;
    // one reverse step at u^n (w = ws (vbar + dtw ubar), vbar^n = damp w); a
    // velocity-Verlet run is the Euler-Cromer recurrence in (u, half-step
    // velocity) between a half kick at its first step and a half kick that
    // forms the full-step velocity it ends with: ws = 1/2 there, and
    // damp = 1 + (1 - dt eta / rho) so that damp ws = 1 - dt eta / (2 rho)
    const double damp_full = A.damp;
    auto reverse_step = [&](const double* un, double dtw, double ws, double damp) {
        A.un = un;
        A.w = T.w;
        A.ubm = T.ubm;
        A.ub_out = T.ub[cb ^ 1];
        A.vb_out = T.vb[cb ^ 1];
        A.damp = damp;
        cudaError_t r;
        if (h->dw) {
            r = launch_adj_mask_publish_dw(T.ub[cb], T.vb[cb], h->bcc, h->bct, dtw, ws,
                                           h->recdw[0], un, h->vol, h->n_pad, 1.0 / h->delta,
                                           T.ubm, T.w, T.rrec, T.wrec, h->stream);
            D.ub_out = A.ub_out;
            D.vb_out = A.vb_out;
            D.damp = damp;
            if (r == cudaSuccess) r = launch_adj_step_dw(D, agrid, 256, h->stream);
        } else {
            r = launch_adj_mask(T.ub[cb], T.vb[cb], h->bcc, h->bct, h->n_pad, dtw, ws, T.ubm, T.w,
                                h->stream);
            if (r == cudaSuccess) r = launch_adj_step(A, agrid, 256, h->stream);
        }
        cb ^= 1;
        return r;
    };
    cudaError_t ke = cudaSuccess;
    if (T.vv && dLdv) ke = reverse_step(T.fin_u, 0.0, 0.5, 1.0 + damp_full);
    for (int64_t k = T.nck - 1; k >= 0 && ke == cudaSuccess; --k) {
        const int64_t start = k * T.C;
        const int64_t len = std::min(T.C, T.N - start);
        // recompute u^start .. u^{start+len-1} from checkpoint k
        h->step = T.step0 + start;
        ke = cudaMemcpyAsync(h->step_ctr, &h->step, sizeof(int64_t), cudaMemcpyHostToDevice,
                             h->stream);
        if (ke == cudaSuccess) ke = cudaStreamSynchronize(h->stream);
        const int cur = (int)(h->step & 1);
        if (ke == cudaSuccess) ke = launch_insert_u(T.ck_u + k * np3, h->n_pad, h->rec[cur], h->stream);
        if (ke == cudaSuccess && h->dw)
            ke = launch_dw_publish(h->rec[cur], h->recdw[cur], h->n_pad, h->dw_origin,
                                   1.0 / h->delta, h->stream);
        if (ke == cudaSuccess)
            ke = cudaMemcpyAsync(h->v, T.ck_v + k * np3, 8 * np3, cudaMemcpyDeviceToDevice, h->stream);
        if (ke == cudaSuccess)
            ke = cudaMemcpyAsync(T.seg, T.ck_u + k * np3, 8 * np3, cudaMemcpyDeviceToDevice, h->stream);
        for (int64_t t = 1; t < len && ke == cudaSuccess; ++t) {
            ke = launch_one(h, 0);
            if (ke == cudaSuccess) ke = launch_advance(h->step_ctr, 1, h->stream);
            h->step += 1;
            if (ke == cudaSuccess)
                ke = launch_extract_u(h->rec[h->step & 1], h->n_pad, T.seg + t * np3, h->stream);
        }
        // reverse through the segment
        for (int64_t t = len - 1; t >= 0 && ke == cudaSuccess; --t) {
            const bool half = T.vv && start + t == 0;
            ke = reverse_step(T.seg + t * np3, h->dt, half ? 0.5 : 1.0,
                              half ? 1.0 + damp_full : damp_full);
        }
    }
    if (h->dw && ke == cudaSuccess)
        ke = launch_adj_merge_dw(T.gcdw, slots, A.dt_rho, T.gc, h->stream);
    h->frozen = false;
    h->drop_graph();
    // restore the final state u^N, v^N
    h->step = T.step0 + T.N;
    if (ke == cudaSuccess)
        ke = cudaMemcpyAsync(h->step_ctr, &h->step, sizeof(int64_t), cudaMemcpyHostToDevice,
                             h->stream);
    if (ke == cudaSuccess) ke = cudaStreamSynchronize(h->stream);
    if (ke == cudaSuccess) ke = launch_insert_u(T.fin_u, h->n_pad, h->rec[h->step & 1], h->stream);
    if (ke == cudaSuccess && h->dw)
        ke = launch_dw_publish(h->rec[h->step & 1], h->recdw[h->step & 1], h->n_pad, h->dw_origin,
                               1.0 / h->delta, h->stream);
    if (ke == cudaSuccess)
        ke = cudaMemcpyAsync(h->v, T.fin_v, 8 * np3, cudaMemcpyDeviceToDevice, h->stream);
    h->damage_fresh = false;
    h->peek_step = -1;
    if (ke != cudaSuccess) return cuda_fail(ke, "adjoint sweep");

    // outputs
    if (dL_dload) {
        PD_CUDA(launch_sum(T.gl, h->n, A.dt_rho, T.partial, T.n_partial, T.out, h->stream),
                "load gradient");
        PD_CUDA(cudaMemcpyAsync(dL_dload, T.out, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                "copy load gradient");
    }
    auto from_lib = [&](const double* src, double* dst) -> pd_status {
        if (!dst) return PD_OK;
        const bool dev = is_device_ptr(dst);
        double* o = dev ? dst : h->staging;
        PD_CUDA(launch_from_lib3(src, h->gid, h->n, o, h->stream), "reorder");
        if (!dev)
            PD_CUDA(cudaMemcpyAsync(dst, h->staging, 24 * h->n, cudaMemcpyDeviceToHost, h->stream),
                    "copy gradient to host");
        PD_CUDA(cudaStreamSynchronize(h->stream), "synchronize");
        return PD_OK;
    };
    if ((st = from_lib(T.ub[cb], dL_du0)) != PD_OK || (st = from_lib(T.vb[cb], dL_dv0)) != PD_OK)
        return st;
    if (dL_dc) {
        std::vector<double> g((size_t)slots);
        PD_CUDA(cudaMemcpyAsync(g.data(), T.gc, 8 * slots, cudaMemcpyDeviceToHost, h->stream),
                "copy stiffness gradient");
        PD_CUDA(cudaStreamSynchronize(h->stream), "synchronize");
        std::vector<int64_t> pos;
        if ((st = canonical_slots(h, pos)) != PD_OK) return st;
        for (size_t s = 0; s < pos.size(); ++s)
            if (pos[s] >= 0) dL_dc[pos[s]] = g[s];
    }
    return check_dev_err(h);
}

pd_status pd_test_tile_wait_extra(pd_handle* h, int32_t bytes)
{
    if (!h) return fail(PD_ERR_ARG, "NULL handle");
    if (!(h->lattice && h->lat_var >= 2))
        return fail(PD_ERR_ARG, "the handle does not use the tile step (lat_variant 2..4)");
    if (bytes < 0 || bytes > 65536) return fail(PD_ERR_ARG, "bytes must be in [0, 65536]");
    h->lat_tma.extra_tx = bytes;
    h->drop_graph();  // captured launches hold the old value
    return PD_OK;
}

pd_status pd_autotune(pd_handle* h, int32_t trial_steps, int32_t* block_threads,
                      int32_t* blocks_per_sm)
{
    NvtxScope nvtx_scope_("pd_autotune");
    if (!h) return fail(PD_ERR_ARG, "NULL handle");
    if (trial_steps < 1 || trial_steps > 1000) return fail(PD_ERR_ARG, "trial_steps in [1, 1000]");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    PD_CUDA(cudaStreamSynchronize(h->stream), "synchronize");
    // save everything a step writes: displacement records and low parts, velocity,
    // bond flags, damage and the step counter
    struct Buf {
        void* dev;
        size_t bytes;
        std::vector<uint8_t> keep;
    };
    const int64_t np = h->n_pad;
    std::vector<Buf> bufs;
    if (h->lattice) {
        for (int k = 0; k < 2; ++k) {
            bufs.push_back({h->lat_u[k], (size_t)(24 * np), {}});
            bufs.push_back({h->lat_pub[k], (size_t)(16 * np), {}});
        }
        bufs.push_back({h->v, (size_t)(12 * np), {}});
        bufs.push_back({h->damage, (size_t)(4 * np), {}});
    } else if (h->precision == 32) {
        bufs.push_back({h->rec32[0], (size_t)(32 * np), {}});
        bufs.push_back({h->rec32[1], (size_t)(32 * np), {}});
        bufs.push_back({h->lo32, (size_t)(16 * np), {}});
        bufs.push_back({h->v, (size_t)(12 * np), {}});
        bufs.push_back({h->damage, (size_t)(4 * np), {}});
    } else {
        bufs.push_back({h->rec[0], (size_t)(64 * np), {}});
        bufs.push_back({h->rec[1], (size_t)(64 * np), {}});
        if (h->dw) {
            bufs.push_back({h->recdw[0], (size_t)(64 * np), {}});
            bufs.push_back({h->recdw[1], (size_t)(64 * np), {}});
        }
        bufs.push_back({h->v, (size_t)(24 * np), {}});
        bufs.push_back({h->damage, (size_t)(8 * np), {}});
    }
    bufs.push_back({h->bits, (size_t)(4 * h->n_slices * h->Q * 32), {}});
    if (h->integ)
        bufs.push_back({h->integ, (size_t)((h->precision == 32 ? 4 : 8) * h->n_slices * h->Q * 32 * 32), {}});
    bufs.push_back({h->step_ctr, 2 * sizeof(int64_t), {}});
    bufs.push_back({h->err, sizeof(int), {}});
    for (Buf& b : bufs) {
        b.keep.resize(b.bytes);
        PD_CUDA(cudaMemcpy(b.keep.data(), b.dev, b.bytes, cudaMemcpyDeviceToHost), "save state");
    }
    auto restore = [&]() -> pd_status {
        for (Buf& b : bufs)
            PD_CUDA(cudaMemcpyAsync(b.dev, b.keep.data(), b.bytes, cudaMemcpyHostToDevice, h->stream),
                    "restore state");
        return PD_OK;
    };
    const int old_block = h->block, old_bps = h->blocks_per_sm, old_var = h->lat_var;
    const int64_t step0 = h->step;
    cudaEvent_t e0, e1;
    PD_CUDA(cudaEventCreate(&e0), "event");
    PD_CUDA(cudaEventCreate(&e1), "event");
    float best = 1e30f;
    int best_block = old_block, best_bps = old_bps, best_var = old_var;
    pd_status st = PD_OK;
    h->drop_graph();
    // bond-based lattice models: the stencil step's compiled variants too (both
    // register budgets; single models also the shared-memory tile shapes, whose
    // block and grid are fixed by the shape)
    const int n_var = !(h->lattice && h->model == 0) ? 1 : h->batch ? 2 : 2 + kLatTmaShapes;
    for (int var = 0; var < n_var && st == PD_OK; ++var)
    for (int block : {128, 256}) {
        if (var >= 2 && block != 256) continue;
        for (int bps = 1; bps <= 16 && st == PD_OK; ++bps) {
            h->lat_var = var;
            h->block = block;
            if ((st = choose_grid(h, bps)) != PD_OK) break;
            if ((st = restore()) != PD_OK) break;
            cudaError_t e = launch_one(h, 0);
            for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) e = launch_one(h, k + 1);
            if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
            for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) e = launch_one(h, k + 1);
            if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "autotune trial");
                break;
            }
            if (ms < best) {
                best = ms;
                best_block = block;
                best_bps = bps;
                best_var = var;
            }
            if (var >= 2) break;  // the tile step's grid does not depend on bps
            int occ = 0;
            const void* fn = step_kernel_fn(h);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, 0);
            if (bps >= occ) break;  // larger requests are capped to the same grid
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->block = st == PD_OK ? best_block : old_block;
    h->blocks_per_sm = st == PD_OK ? best_bps : old_bps;
    h->lat_var = st == PD_OK ? best_var : old_var;
    pd_status st2 = choose_grid(h, h->blocks_per_sm);
    pd_status st3 = restore();
    h->step = step0;
    if (st != PD_OK) return st;
    if (st2 != PD_OK) return st2;
    if (st3 != PD_OK) return st3;
    if (block_threads) *block_threads = h->block;
    if (blocks_per_sm) *blocks_per_sm = h->blocks_per_sm;
    return PD_OK;
}

pd_status pd_set_params(pd_handle* h, double c, double sc, double load, double disp_rate,
                        const double* c_bond)
{
    NvtxScope nvtx_scope_("pd_set_params");
    if (!h) return fail(PD_ERR_ARG, "NULL handle");
    if (h->batch) return fail(PD_ERR_STATE, "pd_set_params is not available on a batch handle");
    if (h->model == 1 && c_bond)
        return fail(PD_ERR_STATE, "per-bond stiffness is not available with the state-based model");
    if (!(c > 0.0) || !std::isfinite(c)) return fail(PD_ERR_ARG, "c must be > 0");
    if (!(sc > 0.0) || !std::isfinite(sc)) return fail(PD_ERR_ARG, "sc must be > 0");
    if (!std::isfinite(load) || !std::isfinite(disp_rate))
        return fail(PD_ERR_ARG, "load and disp_rate must be finite");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    if (c_bond) {
        for (int64_t k = 0; k < h->n_bonds; ++k)
            if (!(c_bond[k] > 0.0) || !std::isfinite(c_bond[k]))
                return fail(PD_ERR_ARG, "c_bond must be finite and > 0");
        std::vector<int64_t> pos;
        pd_status st = canonical_slots(h, pos);
        if (st != PD_OK) return st;
        const size_t slots = pos.size();
        if (!h->cbond) {
            cudaError_t e = h->alloc((uint8_t**)&h->cbond, slots * (h->precision == 32 ? 4 : 8));
            if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc c_bond");
        }
        if (h->precision == 32) {
            std::vector<float> cb(slots, 0.0f);
            for (size_t s = 0; s < slots; ++s)
                if (pos[s] >= 0) cb[s] = (float)c_bond[pos[s]];
            PD_CUDA(cudaMemcpyAsync(h->cbond, cb.data(), slots * 4, cudaMemcpyHostToDevice, h->stream),
                    "upload c_bond");
        } else {
            std::vector<double> cb(slots, 0.0);
            for (size_t s = 0; s < slots; ++s)
                if (pos[s] >= 0) cb[s] = c_bond[pos[s]];
            PD_CUDA(cudaMemcpyAsync(h->cbond, cb.data(), slots * 8, cudaMemcpyHostToDevice, h->stream),
                    "upload c_bond");
            if (h->dw) {
                if (!h->cbdw) {
                    cudaError_t e = h->alloc(&h->cbdw, slots);
                    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc c_bond");
                }
                PD_CUDA(launch_dw_split((const double*)h->cbond, (int64_t)slots, h->cbdw, h->stream),
                        "double-word c_bond");
            }
        }
    }
    const bool pbc = c_bond != nullptr;
    const bool reweight = pbc != h->per_bond_c || (!pbc && c != h->c);
    h->per_bond_c = pbc;
    h->c = c;
    if (h->sc_mode == 0) {
        h->sc = sc;
        h->sc_lo = h->sc_hi = sc;
    }
    h->load = load;
    h->disp_rate = disp_rate;
    h->drop_graph();
    {  // the kernel variant depends on per-bond stiffness
        pd_status st = choose_grid(h, h->blocks_per_sm);
        if (st != PD_OK) return st;
    }
    if (reweight) {
        pd_status st = upload_weights(h);
        if (st != PD_OK) return st;
    }
    PD_CUDA(cudaStreamSynchronize(h->stream), "synchronize");
    h->damage_fresh = false;
    h->peek_step = -1;
    return PD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// pd_adjoint_backward_static: the reverse sweep with its working memory in one
// file-scope device array, for callers that cannot allocate device memory.
// Calls share the array; overlapping calls race (documented in pd.h).

static __device__ __align__(256) unsigned char pd_static_scratch[PD_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
unsigned char* g_static_ptr[kStaticMaxDevices] = {};

// device address of pd_static_scratch on `device` (current), looked up once
pd_status static_scratch(int device, unsigned char** out)
{
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (device < 0 || device >= kStaticMaxDevices)
        return fail(PD_ERR_ARG, "static scratch: device %d out of range", device);
    if (!g_static_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, pd_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_static_ptr[device] = (unsigned char*)p;
    }
    *out = g_static_ptr[device];
    return PD_OK;
}

// the sweep's buffers, carved at 256-byte boundaries from `base` (nullptr: sizing only)
struct StaticBufs {
    double *ub[2], *vb[2], *ubm, *w, *gl, *gc, *partial, *out, *dc;
    int64_t* off;
    int32_t* idx;
};

size_t carve_static(unsigned char* base, int64_t np3, int64_t n_pad, int64_t slots, int n_partial,
                    int64_t n, int64_t n_bonds, bool want_c, bool c_host, StaticBufs& b)
{
    size_t used = 0;
    auto take = [&](size_t bytes) -> unsigned char* {
        const size_t at = (used + 255) & ~(size_t)255;
        used = at + std::max<size_t>(bytes, 8);
        return base ? base + at : nullptr;
    };
    for (int k = 0; k < 2; ++k) b.ub[k] = (double*)take(8 * np3);
    for (int k = 0; k < 2; ++k) b.vb[k] = (double*)take(8 * np3);
    b.ubm = (double*)take(8 * np3);
    b.w = (double*)take(8 * np3);
    b.gl = (double*)take(8 * n_pad);
    b.gc = (double*)take(8 * slots);
    b.partial = (double*)take(8 * (size_t)n_partial);
    b.out = (double*)take(8);
    b.off = want_c ? (int64_t*)take(8 * (n + 1)) : nullptr;
    b.idx = want_c ? (int32_t*)take(4 * n_bonds) : nullptr;
    b.dc = c_host ? (double*)take(8 * n_bonds) : nullptr;
    return used;
}

}  // namespace

extern "C" {

pd_status pd_adjoint_backward_static(pd_handle* h, const double* dLdu, const double* dLdv,
                                     double* dL_dc, double* dL_dload, double* dL_du0,
                                     double* dL_dv0)
{
    NvtxScope nvtx_scope_("pd_adjoint_backward_static");
    if (!h) return fail(PD_ERR_ARG, "NULL handle");
    auto& T = h->tape;
    if (!T.valid) return fail(PD_ERR_STATE, "no recorded adjoint forward run");
    if (!dLdu) return fail(PD_ERR_ARG, "dLdu is required");
    PD_CUDA(cudaSetDevice(h->device), "cudaSetDevice");
    const int64_t np3 = 3 * h->n_pad;
    const int64_t slots = h->n_slices * 32LL * h->Q * 32;
    const int n_partial = sum_partials_needed(h->n);
    const int64_t n_bonds = h->off[(size_t)h->n];
    const bool want_c = dL_dc != nullptr;
    const bool c_host = want_c && !is_device_ptr(dL_dc);
    StaticBufs b{};
    const size_t need = carve_static(nullptr, np3, h->n_pad, slots, n_partial, h->n, n_bonds,
                                     want_c, c_host, b);
    if (need > (size_t)PD_STATIC_SCRATCH_BYTES)
        return fail(PD_ERR_ARG,
                    "pd_adjoint_backward_static: this model needs %zu bytes of scratch, above "
                    "the static maximum of %zu bytes (use pd_adjoint_backward)",
                    need, (size_t)PD_STATIC_SCRATCH_BYTES);
    unsigned char* base = nullptr;
    pd_status st = static_scratch(h->device, &base);
    if (st != PD_OK) return st;
    carve_static(base, np3, h->n_pad, slots, n_partial, h->n, n_bonds, want_c, c_host, b);

    // every buffer starts at zero (gc and gl accumulate; earlier calls leave data)
    PD_CUDA(cudaMemsetAsync(base, 0, need, h->stream), "clear static scratch");
    auto to_lib = [&](const double* src, double* dst) -> pd_status {
        if (!src) return PD_OK;
        const double* s = src;
        if (!is_device_ptr(src)) {
            PD_CUDA(cudaMemcpyAsync(h->staging, src, 24 * h->n, cudaMemcpyHostToDevice, h->stream),
                    "copy gradient to device");
            s = h->staging;
        }
        PD_CUDA(launch_to_lib3(s, h->gid, h->n, dst, h->stream), "reorder");
        PD_CUDA(cudaStreamSynchronize(h->stream), "synchronize");
        return PD_OK;
    };
    if ((st = to_lib(dLdu, b.ub[0])) != PD_OK || (st = to_lib(dLdv, b.vb[0])) != PD_OK) return st;

    int sms = 0;
    PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device), "sm count");
    const int agrid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * 8,
                                                                  (h->n_slices + 7) / 8));
    AdjArgs A{};
    A.x64 = h->x64;
    A.nbr = h->nbr;
    A.bits = h->bits;
    A.sw = h->sw;
    A.Q = h->Q;
    A.vol = h->vol;
    A.cbond = h->per_bond_c ? (const double*)h->cbond : nullptr;
    A.ilen = h->ilen;
    A.c = h->c;
    A.gc = b.gc;
    A.gl = b.gl;
    A.bcc = h->bcc;
    A.bct = h->bct;
    A.dt_rho = h->dt / h->rho;
    A.damp = 1.0 - h->dt * h->eta / h->rho;
    A.n = h->n;

    // segments are recomputed with direct launches (no graph is built or used)
    h->frozen = true;
    int cb = 0;
    // one reverse step at u^n, with the half kicks of a velocity-Verlet run as
    // in pd_adjoint_backward
    const double damp_full = A.damp;
    auto reverse_step = [&](const double* un, double dtw, double ws, double damp) {
        cudaError_t r = launch_adj_mask(b.ub[cb], b.vb[cb], h->bcc, h->bct, h->n_pad, dtw, ws,
                                        b.ubm, b.w, h->stream);
        A.un = un;
        A.w = b.w;
        A.ubm = b.ubm;
        A.ub_out = b.ub[cb ^ 1];
        A.vb_out = b.vb[cb ^ 1];
        A.damp = damp;
        if (r == cudaSuccess) r = launch_adj_step(A, agrid, 256, h->stream);
        cb ^= 1;
        return r;
    };
    cudaError_t ke = cudaSuccess;
    if (T.vv && dLdv) ke = reverse_step(T.fin_u, 0.0, 0.5, 1.0 + damp_full);
    for (int64_t k = T.nck - 1; k >= 0 && ke == cudaSuccess; --k) {
        const int64_t start = k * T.C;
        const int64_t len = std::min(T.C, T.N - start);
        h->step = T.step0 + start;
        ke = cudaMemcpyAsync(h->step_ctr, &h->step, sizeof(int64_t), cudaMemcpyHostToDevice,
                             h->stream);
        if (ke == cudaSuccess) ke = cudaStreamSynchronize(h->stream);
        const int cur = (int)(h->step & 1);
        if (ke == cudaSuccess) ke = launch_insert_u(T.ck_u + k * np3, h->n_pad, h->rec[cur], h->stream);
        if (ke == cudaSuccess && h->dw)
            ke = launch_dw_publish(h->rec[cur], h->recdw[cur], h->n_pad, h->dw_origin,
                                   1.0 / h->delta, h->stream);
        if (ke == cudaSuccess)
            ke = cudaMemcpyAsync(h->v, T.ck_v + k * np3, 8 * np3, cudaMemcpyDeviceToDevice, h->stream);
        if (ke == cudaSuccess)
            ke = cudaMemcpyAsync(T.seg, T.ck_u + k * np3, 8 * np3, cudaMemcpyDeviceToDevice, h->stream);
        for (int64_t t = 1; t < len && ke == cudaSuccess; ++t) {
            ke = launch_one(h, 0);
            if (ke == cudaSuccess) ke = launch_advance(h->step_ctr, 1, h->stream);
            h->step += 1;
            if (ke == cudaSuccess)
                ke = launch_extract_u(h->rec[h->step & 1], h->n_pad, T.seg + t * np3, h->stream);
        }
        for (int64_t t = len - 1; t >= 0 && ke == cudaSuccess; --t) {
            const bool half = T.vv && start + t == 0;
            ke = reverse_step(T.seg + t * np3, h->dt, half ? 0.5 : 1.0,
                              half ? 1.0 + damp_full : damp_full);
        }
    }
    h->frozen = false;
    h->step = T.step0 + T.N;
    if (ke == cudaSuccess)
        ke = cudaMemcpyAsync(h->step_ctr, &h->step, sizeof(int64_t), cudaMemcpyHostToDevice,
                             h->stream);
    if (ke == cudaSuccess) ke = cudaStreamSynchronize(h->stream);
    if (ke == cudaSuccess) ke = launch_insert_u(T.fin_u, h->n_pad, h->rec[h->step & 1], h->stream);
    if (ke == cudaSuccess && h->dw)
        ke = launch_dw_publish(h->rec[h->step & 1], h->recdw[h->step & 1], h->n_pad, h->dw_origin,
                               1.0 / h->delta, h->stream);
    if (ke == cudaSuccess)
        ke = cudaMemcpyAsync(h->v, T.fin_v, 8 * np3, cudaMemcpyDeviceToDevice, h->stream);
    h->damage_fresh = false;
    h->peek_step = -1;
    if (ke != cudaSuccess) return cuda_fail(ke, "adjoint sweep");

    if (dL_dload) {
        PD_CUDA(launch_sum(b.gl, h->n, A.dt_rho, b.partial, n_partial, b.out, h->stream),
                "load gradient");
        PD_CUDA(cudaMemcpyAsync(dL_dload, b.out, sizeof(double), cudaMemcpyDeviceToHost, h->stream),
                "copy load gradient");
    }
    auto from_lib = [&](const double* src, double* dst) -> pd_status {
        if (!dst) return PD_OK;
        const bool dev = is_device_ptr(dst);
        double* o = dev ? dst : h->staging;
        PD_CUDA(launch_from_lib3(src, h->gid, h->n, o, h->stream), "reorder");
        if (!dev)
            PD_CUDA(cudaMemcpyAsync(dst, h->staging, 24 * h->n, cudaMemcpyDeviceToHost, h->stream),
                    "copy gradient to host");
        PD_CUDA(cudaStreamSynchronize(h->stream), "synchronize");
        return PD_OK;
    };
    if ((st = from_lib(b.ub[cb], dL_du0)) != PD_OK || (st = from_lib(b.vb[cb], dL_dv0)) != PD_OK)
        return st;
    if (want_c) {
        PD_CUDA(cudaMemcpyAsync(b.off, h->off.data(), 8 * (h->n + 1), cudaMemcpyHostToDevice,
                                h->stream),
                "copy family offsets");
        if (n_bonds > 0)
            PD_CUDA(cudaMemcpyAsync(b.idx, h->idx.data(), 4 * n_bonds, cudaMemcpyHostToDevice,
                                    h->stream),
                    "copy family");
        PD_CUDA(launch_slots_to_canonical(b.gc, h->nbr, h->gid, b.off, b.idx, h->n, h->Q,
                                          c_host ? b.dc : dL_dc, h->stream),
                "stiffness gradient to canonical order");
        if (c_host && n_bonds > 0)
            PD_CUDA(cudaMemcpyAsync(dL_dc, b.dc, 8 * n_bonds, cudaMemcpyDeviceToHost, h->stream),
                    "copy stiffness gradient");
    }
    return check_dev_err(h);
}

}  // extern "C"
