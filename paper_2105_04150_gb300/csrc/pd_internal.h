// Internal declarations of the peridynamic step library (not installed).
//
// Device layout (nodes in the library's spatial order p = 0..n-1):
//   FP32 path  rec32[2]  ping-pong node records, 2 float4 per node:
//                        {x~, y~, z~, w}  reference position / horizon, centred;
//                                         w = c V_j (constant c) or V_j (per-bond c)
//                        {u~x, u~y, u~z, 0} displacement / horizon (FP32 shadow)
//              u64[2]    ping-pong FP64 displacement, 3 per node (the accumulator)
//              v32       FP32 velocity, 3 per node, updated in place by its owner
//   FP64 path  rec64[2]  ping-pong records, 8 doubles per node {x, y, z, w, ux, uy, uz, 0}
//              v64       FP64 velocity, 3 per node
//   both       nbr       int32 padded family, node p owns nbr[p*W .. p*W+W), W = 32*Q;
//                        member m = q*32 + l sits at p*W + q*32 + l ("q-major"), so
//                        warp lane l reads member q*32+l with one coalesced load;
//                        padding slots hold p itself
//              bits      uint32 bond flags, node p owns bits[p*Q .. p*Q+Q); bit l of word q
//                        is member q*32+l (1 = intact); padding bits are 0
//              bcc       uint8 boundary-condition class per node -> BcClass table
//              gid       int32 caller id of each node
//              x64       FP64 reference coordinates (FP32 path: near-s_c re-test)
//              wsum_inv  1 / sum_j w_j over the family after the initial cuts
//              damage    per node, rewritten by every step
//              step_ctr  int64 device step counter (read by every step kernel)
//              err       int32 device error bits (PD_DEVERR_*)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define PD_DEVERR_NONFINITE 1

namespace pd {

struct BcClass {
    uint32_t mask;     // bit a (0..2): component a displacement-controlled; bit 3: no-fail
    uint32_t pad;
    double disp[3];    // prescribed displacement per unit scale
    double force[3];   // body-force density per unit load
};

struct StepArgsF32 {
    const float4* rec[2];
    double* u64[2];
    float* v;
    const int32_t* nbr;
    uint32_t* bits;
    const float* cbond;        // per slot (n*W) or nullptr
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
    int32_t q_rt;              // Q when the kernel is instantiated for a runtime Q
    int32_t has_nofail;
    int32_t pad0;
    float sc_f, sc_lo_f;       // FP32 copies of sc / sc_lo
    float guard;               // relative band around s_c re-tested in FP64
    float pad1;
    double sc, sc_lo, sc_hi;
    uint64_t sc_seed;
    double dt, eta, rho, disp_rate, load, inv_delta;
};

struct StepArgsF64 {
    const double* rec[2];      // 8 doubles per node
    double* v;
    const int32_t* nbr;
    uint32_t* bits;
    const double* cbond;       // per slot or nullptr
    const uint8_t* bcc;
    const BcClass* bct;
    const int32_t* gid;
    const double* wsum_inv;
    double* damage;
    int* err;
    const int64_t* step_ctr;
    int64_t n;
    int32_t k;
    int32_t q_rt;
    int32_t has_nofail;
    int32_t pad0;
    double sc, sc_lo, sc_hi;
    uint64_t sc_seed;
    double dt, eta, rho, disp_rate, load;
};

// ---- launchers (pd_step_f32.cu / pd_step_f64.cu) --------------------------------
cudaError_t launch_step_f32(const StepArgsF32& a, int Q, int sc_mode, int grid, int block,
                            cudaStream_t s);
cudaError_t launch_step_f64(const StepArgsF64& a, int Q, int sc_mode, int grid, int block,
                            cudaStream_t s);
// kernel entry addresses (occupancy and attribute queries)
const void* step_f32_kernel(int Q, int sc_mode);
const void* step_f64_kernel(int Q, int sc_mode);

// ---- helper kernels (pd_aux.cu) ---------------------------------------------------
cudaError_t launch_advance(int64_t* step_ctr, int64_t k, cudaStream_t s);
// caller-order FP64 arrays <-> internal state
cudaError_t launch_get_state_f32(const double* u64, const float* v32, const int32_t* gid,
                                 int64_t n, double* u_out, double* v_out, cudaStream_t s);
cudaError_t launch_set_state_f32(const double* u_in, const double* v_in, const int32_t* gid,
                                 int64_t n, double inv_delta, double* u64, float4* rec,
                                 float* v32, cudaStream_t s);
cudaError_t launch_get_state_f64(const double* rec64, const double* v64, const int32_t* gid,
                                 int64_t n, double* u_out, double* v_out, cudaStream_t s);
cudaError_t launch_set_state_f64(const double* u_in, const double* v_in, const int32_t* gid,
                                 int64_t n, double* rec64, double* v64, cudaStream_t s);
// damage from the bond flags: phi_p = 1 - sum_alive w_j * wsum_inv_p, written to caller order
cudaError_t launch_damage(int precision, const void* rec, const int32_t* nbr,
                          const uint32_t* bits, const void* wsum_inv, const int32_t* gid,
                          int64_t n, int Q, double* phi_out, cudaStream_t s);
// damage written by the last step (spatial order) -> caller order
cudaError_t launch_gather_damage(int precision, const void* dmg, const int32_t* gid, int64_t n,
                                 double* phi_out, cudaStream_t s);
// node weights w_p (rec .w) and wsum_inv from volumes
// (fam_cnt: members per node after the initial cuts; slots m < fam_cnt[p] are real)
cudaError_t launch_set_weights(int precision, void* rec0, void* rec1, const double* vol,
                               const int32_t* nbr, const int32_t* fam_cnt, int64_t n, int Q,
                               double wscale, void* wsum_inv, cudaStream_t s);

}  // namespace pd
