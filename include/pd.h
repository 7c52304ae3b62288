/*
 * pd.h - C ABI of the GB300-native bond-based peridynamic time stepper.
 *
 * The library advances the explicit, damped time step of a bond-based (PMB)
 * peridynamic model over a fixed neighbour family (arXiv 2105.04150,
 * "PeriPy"): per node it evaluates every intact bond (stretch, Eq. 4), breaks
 * bonds irreversibly at the critical stretch (Eq. 6), reduces the pairwise
 * forces (Eq. 5, Eq. 10), adds the body force, integrates with damped
 * Euler-Cromer (Eq. 11) and applies displacement boundary conditions, and
 * writes the damage (Eq. 8).  All of it runs on one GPU in CUDA kernels.
 *
 * Conventions for every entry point:
 *  - Node ids in and out are the caller's ids 0..n-1; the library keeps its
 *    own spatial order internally and never exposes it.
 *  - "Family" arrays are CSR over the caller's nodes (off[n+1] int64,
 *    idx[off[n]] int32), rows sorted ascending; per-bond arrays
 *    (stiffness, bond flags) follow that CSR order ("canonical order").
 *  - Vectors are row-major n x 3 (x, y, z per node), double unless stated.
 *  - The library copies every input; the caller owns every buffer it passes.
 *  - Pointers documented as "host or device" are classified with
 *    cudaPointerGetAttributes; all other pointers are host pointers.
 *  - Every call returns a pd_status; nothing aborts, traps or exits.  On
 *    error pd_last_error() returns a message (thread-local, valid until the
 *    next call from the same thread).
 *  - Work is queued on the handle's stream (pd_config.stream, or a stream the
 *    library creates); calls that return data to the host synchronise it.
 */
#ifndef PD_H
#define PD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pd_handle pd_handle;

typedef enum {
    PD_OK = 0,
    PD_ERR_ARG = 1,               /* invalid argument (message says which) */
    PD_ERR_CUDA = 2,              /* a CUDA runtime call failed */
    PD_ERR_OOM = 3,               /* device or host allocation failed */
    PD_ERR_NONFINITE = 4,         /* a displacement became NaN/Inf during stepping */
    PD_ERR_UNSTABLE_DT = 5,       /* dt exceeds the explicit stability bound */
    PD_ERR_FAMILY_TOO_LARGE = 6,  /* a family exceeds PD_MAX_FAMILY members */
    PD_ERR_TIMEOUT = 7,           /* reserved for bounded device waits */
    PD_ERR_STATE = 8              /* call not valid in the handle's current state */
} pd_status;

#define PD_PREC_F64 64   /* FP64 throughout */
#define PD_PREC_F32 32   /* FP32 bond arithmetic; an FP64 re-test of bonds whose
                            stretch is near s_c.  Each node's displacement is
                            accumulated in FP64 on lattice models (layout
                            PD_LAYOUT_LATTICE; the bond arithmetic reads it rounded
                            to FP32), else as a float-float pair (48-bit
                            significand, exact two-sum updates; neighbours read the
                            high word and a bf16 rounding of the low word) */
#define PD_PREC_DW 48    /* FP64-grade step from FP32 double-word arithmetic: node
                            state (u, v) and integration in FP64 exactly as with
                            PD_PREC_F64; every bond quantity (xi, eta, y, the
                            stretch of Eq. 4, |y|, the force of Eq. 5) carried as an
                            unevaluated sum of two FP32 numbers (~48-bit significand,
                            bond-force relative error ~1e-13), and the break test
                            decided against the FP64 s_c.  Everything PD_PREC_F64
                            offers: both integrators, per-bond stiffness,
                            softening, batches, the state-based model and the
                            adjoint, which runs in double-word arithmetic
                            as well (see pd_adjoint_forward).
                            pd_get_info reports 48. */
#define PD_MAX_FAMILY 1024
#define PD_MAX_BC_CLASSES 256

typedef struct {
    int32_t precision;    /* PD_PREC_F64, PD_PREC_F32 or PD_PREC_DW */
    int32_t graph_steps;  /* steps per captured CUDA graph; 0 = direct launches */
    double dt;            /* time step, s */
    double damping;       /* eta of Eq. 11, kg m^-3 s^-1 */
    double density;       /* rho, kg m^-3 */
    int32_t check_dt;     /* 1 = refuse a dt above the bound of Silling & Askari (2005) */
    int32_t device;       /* CUDA device ordinal */
    void* stream;         /* cudaStream_t to queue work on; NULL = library-owned stream */
    int32_t block_threads;/* threads per block of the step kernel; 0 = default (256) */
    int32_t blocks_per_sm;/* resident blocks per SM for the step grid; 0 = default */
    int32_t reorder;      /* 0 = keep the caller's node order (best for lattices given
                             row-major); 1 = sort nodes by horizon-sized cells */
    int32_t integrator;   /* PD_INTEGRATOR_EC (0) or PD_INTEGRATOR_VV (1), see below */
    int32_t general;      /* 0 = the regular-lattice stencil step where it applies (see
                             pd_info_t.layout); 1 = always the general sliced-ELL step */
    int32_t lat_variant;  /* compiled variant of the stencil step (lattice handles; the
                             same results bit for bit, pd_autotune searches them):
                             0 = default, records read through L1 (64 registers);
                             1 = the same for 3 resident blocks (80 registers);
                             2, 3, 4 = records staged in shared memory by one TMA
                             bulk tensor copy per block of 16x2x8, 8x4x8 or 32x2x4
                             nodes (z, y, x), single bond-based models only.
                             PD_ERR_ARG for other values or models */
} pd_config;

/*
 * Time integrators (Section 3.6, "Time integration"), with F(u) the force
 * density of Eq. 10 plus the body force:
 *  PD_INTEGRATOR_EC  damped Euler-Cromer (Eq. 11):
 *                    v^{n+1} = v^n + dt (F(u^n) - eta v^n) / rho,
 *                    u^{n+1} = u^n + dt v^{n+1}
 *  PD_INTEGRATOR_VV  damped velocity-Verlet, the damping force taken at the
 *                    half-step velocity (Groot & Warren 1997, lambda = 1/2):
 *                    u^{n+1} = u^n + dt v^n + dt^2/2 a^n,
 *                    vt = v^n + dt/2 a^n,
 *                    a^{n+1} = (F(u^{n+1}) - eta vt) / rho,
 *                    v^{n+1} = v^n + dt/2 (a^n + a^{n+1}),
 *                    a^0 = (F(u^0) - eta v^0) / rho at the state last set (or 0).
 *                    pd_get_state returns the full-step v^n (one extra force
 *                    evaluation that changes nothing); pd_set_state starts a new
 *                    history (a^n is formed again from the state given).
 * One step costs the same in both (one force evaluation).
 */
#define PD_INTEGRATOR_EC 0
#define PD_INTEGRATOR_VV 1

typedef struct {
    double c;             /* micromodulus, Eq. 5 (see pd_micromodulus) */
    double sc;            /* critical stretch, used when sc_mode == 0 */
    int32_t sc_mode;      /* 0 = constant sc; 1 = per-bond draw U[sc_lo, sc_hi) */
    int32_t model;        /* 0 = bond-based PMB (c); 1 = ordinary state-based linear
                             solid (bulk_modulus, shear_modulus), see below */
    uint64_t sc_seed;     /* sc_mode 1: SplitMix64 seed; bond {i,j} uses output
                             min(i,j)*2^32 + max(i,j) + 1 of the stream (caller ids) */
    double sc_lo, sc_hi;
    double kr;            /* 0 = PMB (Eq. 5-6); >= 1 = bilinear softening, see below */
    double bulk_modulus;  /* model 1: K (Pa) */
    double shear_modulus; /* model 1: G (Pa) */
    double kink_ratio;    /* kr >= 1: 0 = bilinear; > 1 = trilinear with the kink at
                             s_1 = kink_ratio * s_0 (< s_c) */
    double kink_force;    /* trilinear: force at the kink / peak force c s_0, in (0, 1] */
} pd_material;

/*
 * Ordinary state-based model (model = 1; the paper's "State-based
 * Peridynamics" section: a nodal dilation loop, then the force loop), with the
 * linear peridynamic solid of Silling et al. (2007) and a constant influence
 * function: m_i = sum_j |xi|^2 V_j, theta_i = (3/m_i) sum_j mu_ij |xi| e_ij V_j
 * (e = |y| - |xi|), t_ij = (3 K theta_i / m_i)|xi| + (15 G / m_i)(e - theta_i |xi|/3),
 * F_i = sum_j mu_ij (t_ij + t_ji) V_j y/|y|.  Bonds break as in Eq. 6.  Unlike
 * the PMB law it is not limited to Poisson's ratio 1/4.  FP64, FP32 and
 * PD_PREC_DW handles (FP32 and PD_PREC_DW: the bond-based path's records,
 * horizon units and near-s_c FP64 decision) with either integrator;
 * c is not used (any value > 0) except by the dt stability check;
 * in batches with one (K, G) for every instance; no softening, per-bond
 * stiffness or adjoint.  Two kernels per step.
 */

/*
 * Bilinear softening (Section 6, Example 3: the damage model with linear
 * elastic limit s_0 and k_r = s_c / s_0 = G_F / G_0, s_0 = sqrt(5 G_0 / (6 E delta))):
 * with kr >= 1 every bond has s_0 = s_c / kr and an integrity
 *   mu = 1                                    while its stretch never exceeded s_0,
 *   mu = s_0 (s_c - k) / (k (s_c - s_0))      k = the largest stretch so far (< s_c),
 *   mu = 0                                    once k >= s_c (broken, as in Eq. 6),
 * and pulls with c s mu V_j (Eq. 5 times mu): the force rises to c s_0, falls
 * linearly to zero at s_c, and unloads along the secant to the origin.  With
 * kink_ratio > 1 the law is trilinear (Section 6, Example 2): the force falls
 * from c s_0 to kink_force * c s_0 at s_1 = kink_ratio * s_0, then to zero at
 * s_c; mu = envelope(k) / (c k).  The damage (Eq. 8) weighs each bond by its
 * integrity.  kr = 1 is the PMB law.
 * Not available with the adjoint; in a batch, kr, kink_ratio and kink_force
 * must be the same for every instance.
 */
typedef struct {
    const uint8_t* type;   /* n*3: 1 = displacement-controlled component, 0 = free */
    const double* disp;    /* n*3: prescribed displacement per unit scale (NULL = 0) */
    const double* force;   /* n*3: body-force density per unit load, N m^-3 (NULL = 0) */
    const uint8_t* no_fail;/* n: bonds touching a flagged node never break (NULL = none) */
    double disp_rate;      /* displacement scale rate, see ramp_steps */
    double load;           /* body-force scale */
    int64_t ramp_steps;    /* 0: the displacement scale after step k is disp_rate * k;
                              T > 0: smooth start (Sections 5-6, a fifth-order
                              displacement-time curve with zero initial velocity and
                              acceleration): disp_rate * T * P(k/T) for k < T with
                              P(t) = t^4 - (3/5) t^5, then disp_rate * (k - 3T/5) */
} pd_bc;

typedef struct {
    int64_t n;            /* nodes */
    int64_t n_bonds;      /* directed bonds in the family after the initial cuts */
    int64_t step;         /* steps taken so far (index of the next step) */
    int32_t precision;
    int32_t ell_width;    /* padded family width used on the device (multiple of 32) */
    int64_t device_bytes; /* device memory held by the handle */
    int32_t layout;       /* PD_LAYOUT_SELL, or PD_LAYOUT_LATTICE: an FP32 Euler-Cromer
                             PMB model with uniform volumes, a linear loading ramp and
                             the caller's node order allowed (reorder 0), whose nodes
                             fill a cubic lattice box and whose family is the
                             122-offset stencil (3 dx <= delta < sqrt(10) dx) minus
                             cuts; its steps run the lattice stencil kernel (no
                             neighbour ids read; u accumulated in FP64, published to
                             the bond arithmetic rounded to FP32) */
    int32_t step_registers; /* registers per thread of the step kernel the handle
                               launches (after pd_autotune: the variant it chose) */
    int32_t lat_variant;    /* lattice handles: the stencil step's variant in use
                               (pd_config.lat_variant); else 0 */
} pd_info_t;
#define PD_LAYOUT_SELL 0
#define PD_LAYOUT_LATTICE 1

/*
 * pd_micromodulus - c = 18 K / (pi delta^4) (Eq. 5, Section 2.2).
 * K: bulk modulus (Pa), delta: horizon (m).  PD_ERR_ARG unless both > 0.
 */
pd_status pd_micromodulus(double K, double delta, double* c_out);

/*
 * pd_critical_stretch - the critical stretch of Eq. 7 from the fracture energy
 * release rate G_F (J/m^2), Young's modulus E (Pa; E = 3 K (1 - 2 nu)) and the
 * horizon delta (m), for a three-dimensional body or a plane-stress or
 * plane-strain two-dimensional one:
 *   PD_DIM_3D        s_c = sqrt(5 G_F / (6 E delta))
 *   PD_PLANE_STRESS  s_c = sqrt(4 pi G_F / (9 E delta))
 *   PD_PLANE_STRAIN  s_c = sqrt(5 pi G_F / (12 E delta))
 * Host-only.  PD_ERR_ARG unless G_F, E and delta are finite and > 0 and dim is
 * one of the three.
 */
#define PD_PLANE_STRESS 1
#define PD_PLANE_STRAIN 2
#define PD_DIM_3D 3
pd_status pd_critical_stretch(double G_F, double E, double delta, int32_t dim, double* s_c_out);

/*
 * pd_stiffness_factors - stiffness corrections as per-bond factors, one per
 * directed bond of the family (fam_off[n+1], fam_idx: canonical order, e.g.
 * from pd_get_family), to pass as c_bond = c * factor to pd_set_params:
 *   PD_STIFF_CONICAL  conical micromodulus c(|xi|) = c1 (1 - |xi|/delta)
 *                     (Section 2.2, micromodulus functions); equating the strain
 *                     energy density under uniform dilation with (9/2) K eps^2
 *                     gives c1 = 90 K / (pi delta^4) = 5 c, so the factor is
 *                     5 (1 - |xi|/delta)
 *   PD_STIFF_SURFACE  volume surface correction lambda_ij = 2 V0 / (V_i + V_j)
 *                     ("Surface correction factors"), V_i = sum over the family
 *                     of node i of V_j, and v0 > 0 the family volume of a node in
 *                     the bulk (on a cubic lattice with delta = 3.01 dx that is
 *                     122 dx^3)
 *   PD_STIFF_PARTIAL  partial volume beta_ij of the discrete equation of motion
 *                     (Section 2.3): the fraction of node j's cell inside the
 *                     horizon, by the linear rule (horizon + dx/2 - |xi|) / dx
 *                     clipped to [0, 1], dx > 0 the lattice spacing; build the
 *                     family with horizon + dx/2 to include the cells that
 *                     straddle the horizon from outside
 * The flags combine (the factors multiply).  coords n*3, volumes n (host);
 * factor: host, one double per family entry.  Host-only work.  PD_ERR_ARG on
 * bad flags, horizon, v0, dx or family.
 */
#define PD_STIFF_CONICAL 1
#define PD_STIFF_SURFACE 2
#define PD_STIFF_PARTIAL 4
pd_status pd_stiffness_factors(int64_t n, const double* coords, const double* volumes,
                               double horizon, const int64_t* fam_off, const int32_t* fam_idx,
                               int32_t flags, double v0, double dx, double* factor);

/*
 * pd_create - build a model and upload it to the GPU.
 *  n        nodes (>= 1, < 2^31)
 *  coords   host, n*3 reference positions x_i (m)
 *  volumes  host, n nodal volumes dV_i (> 0)
 *  horizon  delta (m) of the family H_i = { j != i : |x_i - x_j| <= delta } (Eq. 9)
 *  fam_off, fam_idx  host CSR family in canonical order, or both NULL to let
 *           the library search it (uniform cell grid, inclusive distance test)
 *  cuts     host, n_cuts*6 doubles {axis, pos, lo_a, hi_a, lo_b, hi_b}: planar
 *           rectangles x[axis] = pos, lo_a <= x[a] <= hi_a, lo_b <= x[b] <= hi_b
 *           ((a, b) = the other axes ascending).  A bond whose segment crosses a
 *           rectangle is removed before the first step (initial notch, Section 6).
 *  mat, bc, cfg  see the structs; all required.
 *  out      receives the handle.
 * Returns PD_ERR_ARG for invalid sizes, non-finite inputs, non-positive volumes,
 * more than PD_MAX_BC_CLASSES distinct (type, disp, force, no_fail) tuples;
 * PD_ERR_FAMILY_TOO_LARGE when a family exceeds PD_MAX_FAMILY;
 * PD_ERR_UNSTABLE_DT when cfg->check_dt is set and dt is too large;
 * PD_ERR_OOM / PD_ERR_CUDA on allocation or runtime failure (nothing leaks).
 * The initial state is u = v = 0 with every bond of the family intact, step 0.
 */
pd_status pd_create(int64_t n, const double* coords, const double* volumes, double horizon,
                    const int64_t* fam_off, const int32_t* fam_idx,
                    const double* cuts, int32_t n_cuts,
                    const pd_material* mat, const pd_bc* bc, const pd_config* cfg,
                    pd_handle** out);

/* pd_destroy - release every resource of the handle (NULL is ignored). */
void pd_destroy(pd_handle* h);

/* pd_last_error - message of the last failed call on this thread ("" if none). */
const char* pd_last_error(void);

/* pd_get_info - sizes and step counter of the handle. */
pd_status pd_get_info(pd_handle* h, pd_info_t* out);

/*
 * pd_get_family - the family after the initial cuts, canonical CSR order.
 * off: host int64[n+1]; idx: host int32[n_bonds] (idx may be NULL to get off only).
 */
pd_status pd_get_family(pd_handle* h, int64_t* off, int32_t* idx);

/*
 * pd_step - advance n_steps damped Euler-Cromer steps (Eqs. 4-6, 8, 10-11):
 * per step one fused kernel evaluates all intact bonds, breaks those with
 * s >= s_c for good (no force from a bond in the step it breaks, Algorithm
 * bond_index), reduces F_i, adds load * force_i, updates
 * v <- v + dt (F - eta v) / rho and u <- u + dt v, overwrites controlled
 * components with u = disp * disp_rate * (k+1), v = disp * disp_rate / dt,
 * and writes the damage.  Asynchronous on the handle's stream; a non-finite
 * displacement is reported by the next synchronising call (PD_ERR_NONFINITE).
 * n_steps >= 0.  Whole groups of pd_config.graph_steps steps replay one CUDA
 * graph (its kernels read the device step counter, one advance per graph);
 * the rest are direct launches: on FP32 lattice handles one launch per step
 * (two for the state-based model) whose kernel sets the counter itself, on
 * the others the step kernels and one counter advance.
 */
pd_status pd_step(pd_handle* h, int64_t n_steps);

/* pd_sync - wait for queued work and report device-side errors. */
pd_status pd_sync(pd_handle* h);

/*
 * pd_get_state / pd_set_state - displacement and velocity (n*3 doubles each,
 * host or device, either may be NULL) and the step counter (host, may be NULL).
 * pd_set_state also accepts step < 0 to keep the current counter.
 */
pd_status pd_get_state(pd_handle* h, double* u, double* v, int64_t* step);
pd_status pd_set_state(pd_handle* h, const double* u, const double* v, int64_t step);

/*
 * pd_get_bonds / pd_set_bonds - bond flags mu (1 intact, 0 broken), one byte per
 * directed bond in canonical order (host).  pd_set_bonds rejects values other than 0/1.
 */
pd_status pd_get_bonds(pd_handle* h, uint8_t* mu);

/*
 * pd_get_bond_integrity - each directed bond's integrity mu in [0, 1] (canonical
 * order, host doubles): the bilinear-softening factor above, or 1 / 0 for an
 * intact / broken bond of the PMB law.
 */
pd_status pd_get_bond_integrity(pd_handle* h, double* mu);
/* (With bilinear softening, pd_set_bonds also restarts every bond's history:
 * integrity 1 for the bonds it marks intact, 0 for the others.) */
pd_status pd_set_bonds(pd_handle* h, const uint8_t* mu);

/*
 * pd_remove_bonds - break m bonds after creation, e.g. to cut a notch or a
 * pre-crack into a model built without one: the notched beams of Section 6
 * break every bond crossing the notch's void as an initial condition, and a
 * broken bond carries no force for the rest of the run (Eq. 6).  pairs: host,
 * 2*m int64 node ids (i, j) in the caller's order (the concatenated ids of a
 * batch); both directions i->j and j->i are broken.  Every pair must be a bond
 * of the family after the initial cuts; nothing changes if one is not
 * (PD_ERR_ARG names it).  Unlike an initial cut, a removed bond stays in the
 * family, so it counts as broken in pd_damage (Eq. 8).  With bilinear
 * softening the integrity of the removed bonds becomes 0.  Synchronises the
 * handle's stream; m = 0 does nothing.
 */
pd_status pd_remove_bonds(pd_handle* h, const int64_t* pairs, int64_t m);

/*
 * pd_damage - phi_i = 1 - sum_j mu_ij V_j / sum_j V_j over the family after the
 * initial cuts (Eq. 8), for the current state.  phi: n doubles, host or device.
 */
pd_status pd_damage(pd_handle* h, double* phi);

/*
 * pd_set_params - change material and load without rebuilding the model
 * (Section 3.6, "Running simulations").  c > 0, sc > 0, load and disp_rate
 * finite.  sc applies to sc_mode 0.  c_bond: host, per directed bond in
 * canonical order (> 0, symmetric between i->j and j->i), or NULL for the
 * constant c.
 */
pd_status pd_set_params(pd_handle* h, double c, double sc, double load, double disp_rate,
                        const double* c_bond);

/* ---------------------------------------------------------------------------
 * Sensitivities (outer-loop use, Section 3.6): the gradient of a loss of the
 * final state with respect to every directed bond's stiffness, the body-force
 * load and the initial state, by a hand-written reverse sweep of the damped
 * Euler-Cromer recurrence or of the damped velocity-Verlet run (the handle's
 * integrator; the time-integration equations of Section 2.4).  FP64 and
 * PD_PREC_DW PMB handles without softening (PD_ERR_STATE otherwise), not batch
 * handles.  A velocity-Verlet run must start where the state was set
 * (pd_set_state, or creation), so that its acceleration is formed afresh from
 * (u^0, v^0); then dL_dv0 is the derivative with respect to that velocity and
 * dLdv refers to the full-step velocity v^N that pd_get_state reports.  On PD_PREC_DW handles the recorded and
 * recomputed forward runs use the double-word step and pd_adjoint_backward's
 * reverse sweep is in double-word arithmetic too (FP64-grade; the same outputs
 * to ~1e-10); pd_adjoint_backward_static keeps the FP64 reverse sweep.
 *
 * pd_adjoint_forward - advance n_steps (>= 1) from the current state with the
 *   bond flags frozen (no bond breaks, so the run is a smooth function of the
 *   parameters) and record (u, v) every checkpoint_every steps (0 = ceil(sqrt(
 *   n_steps))) on the device.  Afterwards the state is u^N, v^N as for pd_step.
 *   Device memory: ceil(N/C) * 48 B + C * 24 B per node.
 *
 * pd_adjoint_backward - given dL/du^N and dL/dv^N (n*3 doubles, host or device;
 *   dLdv may be NULL = 0) of the last pd_adjoint_forward, run the reverse sweep
 *   (each segment of C steps is recomputed forward from its checkpoint) and
 *   write any of: dL_dc (host, per directed bond in canonical order: the
 *   derivative with respect to the stiffness of the entry i->j, which enters
 *   only F_i; an undirected bond's sensitivity is the sum of its two entries),
 *   dL_dload (host scalar), dL_du0 / dL_dv0 (n*3, host or device).  The handle's
 *   state is left at u^N, v^N.  PD_ERR_STATE without a recorded forward.
 */
pd_status pd_adjoint_forward(pd_handle* h, int64_t n_steps, int64_t checkpoint_every);
pd_status pd_adjoint_backward(pd_handle* h, const double* dLdu, const double* dLdv,
                              double* dL_dc, double* dL_dload, double* dL_du0, double* dL_dv0);

/*
 * pd_adjoint_backward_static - the same reverse sweep, arguments, outputs and
 * errors as pd_adjoint_backward (dL_dc may here also be a device pointer), for
 * callers that cannot allocate device memory when they need the gradient: code
 * whose device memory is owned by another allocator (a framework's memory pool
 * that has reserved the device), and code that must not trigger the implicit
 * device synchronisation that cudaMalloc / cudaFree may cause.  The paper has no
 * counterpart; it is a deployment variant of the entry point above.
 *
 * It allocates nothing: the reverse sweep's working memory (adjoint vectors,
 * per-slot stiffness gradients, the reduction partials of dL_dload, the
 * canonical family for the dL_dc scatter) is carved from one file-scope device
 * array of PD_STATIC_SCRATCH_BYTES (64 MiB) per device, instead of the buffers
 * pd_adjoint_backward allocates on its first call and keeps in the handle.  The
 * array occupies that much device memory wherever the library's device code is
 * loaded.  A model needing more gets PD_ERR_ARG with the required size in
 * pd_last_error().  The need is 152 B per node (node count padded to a
 * multiple of 32) + 8 B per SELL slot; with dL_dc, 8 B per node + 4 B per
 * directed bond more (the family in canonical order), and a further 8 B per
 * directed bond when dL_dc is host memory (each part rounded up to 256 B).  The recorded forward run
 * (pd_adjoint_forward, which does allocate) must exist: PD_ERR_STATE otherwise.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it; make that
 * first call before any stream capture.  Every call, from every handle on the
 * device, shares the one array: each call clears the part it uses before use,
 * and calls whose GPU work overlaps (on different streams, or from different
 * host threads) race on it and give wrong results; serialise them.
 */
#define PD_STATIC_SCRATCH_BYTES (64u << 20)
pd_status pd_adjoint_backward_static(pd_handle* h, const double* dLdu, const double* dLdv,
                                     double* dL_dc, double* dL_dload, double* dL_du0,
                                     double* dL_dv0);

/* ---------------------------------------------------------------------------
 * Batched multi-instance form (outer-loop use: sensitivity, uncertainty
 * quantification, optimisation; Section 3.6 "Running simulations").
 */
typedef struct {
    int64_t n;               /* nodes of this instance (>= 1) */
    const double* coords;    /* host, n*3 */
    const double* volumes;   /* host, n */
    double horizon;          /* delta of this instance (its family is searched alone) */
    const double* cuts;      /* host, n_cuts*6 (see pd_create), or NULL */
    int32_t n_cuts;
    int32_t reserved;
    pd_material mat;         /* c and critical stretch of this instance (the softening
                                parameters, the model and, for the state-based model,
                                bulk_modulus and shear_modulus must equal instance 0's) */
    pd_bc bc;                /* BCs of this instance; disp_rate and load must be equal
                                across the batch (they are handle-wide) */
} pd_instance;

/*
 * pd_batch_create - n_inst independent models advanced together: one handle,
 * one fused launch per step over all instances (no bond joins two instances).
 * Node k of instance b has the batch-wide id node_offset[b] + k in every other
 * call (pd_get_state, pd_damage, pd_get_bonds, ...), node offsets being the
 * prefix sums of the instances' n.  The per-bond s_c draw of an instance with
 * sc_mode 1 is keyed on its own node ids, so an instance behaves exactly as
 * the same model created alone.  dt, damping, density, precision and graph
 * settings come from cfg and are shared.  pd_set_params is not available on a
 * batch handle (PD_ERR_STATE).  Errors as pd_create, plus PD_ERR_ARG when
 * instances disagree on disp_rate/load, or n_inst < 1.
 */
pd_status pd_batch_create(int32_t n_inst, const pd_instance* inst, const pd_config* cfg,
                          pd_handle** out);

/* pd_batch_offsets - node_offset[n_inst+1] (host) of a batch handle (or [0, n] otherwise). */
pd_status pd_batch_offsets(pd_handle* h, int32_t* n_inst, int64_t* node_offset);

/*
 * pd_autotune - time `trial_steps` steps for each candidate launch shape
 * (threads per block 128 or 256, resident blocks per SM up to the kernel's
 * occupancy) and, on bond-based lattice models (PD_LAYOUT_LATTICE), for each
 * compiled variant of the stencil step (pd_config.lat_variant: both register
 * budgets; on single models also the three shared-memory tile shapes, whose
 * launch shape is fixed), and keep the fastest.  The model state (u, v, bond
 * flags, step counter) is saved before and restored after, so the simulation
 * is unchanged.  trial_steps in [1, 1000].  pd_info_t.step_registers and
 * pd_info_t.lat_variant tell the variant kept.
 */
/*
 * Test hook of the tile step's bounded wait (lat_variant 2..4): the barrier of
 * every block's tile copy then waits for `bytes` more than the copy delivers,
 * so the wait runs out (after about 0.5 s, then once more), the block leaves
 * without updating its nodes and the next synchronising call returns
 * PD_ERR_TIMEOUT; pd_set_state clears the error.  bytes = 0 restores the step.
 * PD_ERR_ARG on handles not using the tile step or bytes outside [0, 65536].
 * Host-only (takes effect from the next step launched).
 */
pd_status pd_test_tile_wait_extra(pd_handle* h, int32_t bytes);

pd_status pd_autotune(pd_handle* h, int32_t trial_steps, int32_t* block_threads,
                      int32_t* blocks_per_sm);

#ifdef __cplusplus
}
#endif

#endif /* PD_H */
