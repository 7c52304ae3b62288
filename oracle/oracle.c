/*
 * FP64 CPU oracle for the bond-based (PMB) peridynamic explicit time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * Written from the paper ("PeriPy - A High Performance OpenCL Peridynamics
 * Package", arXiv 2105.04150), plain and slow on purpose:
 *   - family            Eq. (9), Section 2.3
 *   - stretch           Eq. (4), Section 2.2
 *   - PMB force, c      Eq. (5), Section 2.2 (c = 18K / (pi delta^4))
 *   - breaking (mu)     Eq. (6), Section 2.2, and Algorithm "bond_index"
 *                       (the break check comes before the force, a bond that
 *                       breaks contributes nothing in that step)
 *   - discrete EoM      Eqs. (10)-(11), Section 2.3 (beta = 1, no corrections)
 *   - damage            Eq. (8), Section 2.2
 *   - initial notch     Section 6 (bonds crossing the void broken at start)
 *   - damped Euler-Cromer: named only (Section 3.6); read as
 *       v^{n+1} = v^n + dt (F(u^n) - eta v^n) / rho,  u^{n+1} = u^n + dt v^{n+1}
 *   - displacement BC:  u = g * rate * (n+1) after the update, and the velocity
 *       of that component is the prescribed rate g * rate / dt.
 *   - critical stretch  Eq. (7), Section 2.2 (3D, plane stress, plane strain)
 *   - reverse mode      of the damped Euler-Cromer run (or_adjoint) and of the
 *       damped velocity-Verlet run (or_adjoint_vv), bond flags frozen: the
 *       forward assignments reversed in turn (the paper's outer loops,
 *       Section 3.6; it prints no adjoint)
 * Per node the bonds are visited in ascending neighbour id; each node owns its
 * row of bond flags, so the node loop may run in parallel without races.
 *
 * Per-bond critical stretch (an input the paper does not fix): a counter-based
 * SplitMix64 draw (Steele, Lea & Flood 2014) keyed on the unordered pair of
 * caller node ids, mapped to U[lo, hi) with 53 bits.
 *
 * Every function here is pinned by CPU tests against closed forms, invariants
 * or brute force (see the module docstring of oracle/__init__.py for the list).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Number of OpenMP threads of the oracle's loops (CPU-baseline timing). */
#ifdef _OPENMP
#include <omp.h>
#endif
void or_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : 1);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* Eq. (5): constant micromodulus of the PMB model, c = 18 K / (pi delta^4). */
double or_micromodulus(double bulk_modulus, double delta)
{
    double d4 = delta * delta * delta * delta;
    return 18.0 * bulk_modulus / (M_PI * d4);
}

/* Eq. (7), 3D case: s_c = sqrt(5 G_F / (6 E delta)). */
double or_critical_stretch_3d(double G_F, double E, double delta)
{
    return sqrt(5.0 * G_F / (6.0 * E * delta));
}

/* Eq. (7), the two-dimensional cases: plane stress s_c = sqrt(4 pi G_F / (9 E delta)),
 * plane strain s_c = sqrt(5 pi G_F / (12 E delta)). */
double or_critical_stretch_2d(double G_F, double E, double delta, int plane_strain)
{
    if (plane_strain) return sqrt(5.0 * M_PI * G_F / (12.0 * E * delta));
    return sqrt(4.0 * M_PI * G_F / (9.0 * E * delta));
}

/* Young's modulus from the bulk modulus and Poisson's ratio, E = 3 K (1 - 2 nu)
 * (the relation quoted with Eq. 7). */
double or_youngs_modulus(double K, double nu)
{
    return 3.0 * K * (1.0 - 2.0 * nu);
}

/* SplitMix64: the m-th output (m >= 1) of the generator seeded with `seed`. */
uint64_t or_splitmix64(uint64_t seed, uint64_t m)
{
    uint64_t z = seed + m * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Critical stretch of the bond {i, j}: U[lo, hi) from output (key + 1), where
 * key = min(i,j) * 2^32 + max(i,j).  Symmetric in i and j by construction. */
double or_sc_bond(uint64_t seed, double lo, double hi, int64_t i, int64_t j)
{
    uint64_t a = (uint64_t)(i < j ? i : j);
    uint64_t b = (uint64_t)(i < j ? j : i);
    uint64_t key = (a << 32) | b;
    uint64_t h = or_splitmix64(seed, key + 1ULL);
    double unit = (double)(h >> 11) * (1.0 / 9007199254740992.0);
    return lo + (hi - lo) * unit;
}

static double dist2(const double* a, const double* b)
{
    double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
    return dx * dx + dy * dy + dz * dz;
}

/* ------------------------------------------------------------------ */
/* Eq. (9): H_i = { j != i : |x_i - x_j| <= delta }, by brute force, O(n^2).
 * Rows `rows[r]` (or 0..n-1 when rows == NULL).  First call with idx == NULL
 * fills off[0..nrows] (returns total count); the second call fills idx. */
int64_t or_family_bruteforce(const double* x, int64_t n, double delta,
                             const int64_t* rows, int64_t nrows,
                             int64_t* off, int32_t* idx)
{
    double d2 = delta * delta;
    if (idx == NULL) {
        off[0] = 0;
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t i = rows ? rows[r] : r;
            int64_t cnt = 0;
            for (int64_t j = 0; j < n; ++j)
                if (j != i && dist2(x + 3 * i, x + 3 * j) <= d2) ++cnt;
            off[r + 1] = off[r] + cnt;
        }
        return off[nrows];
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows ? rows[r] : r;
        int64_t p = off[r];
        for (int64_t j = 0; j < n; ++j)
            if (j != i && dist2(x + 3 * i, x + 3 * j) <= d2) idx[p++] = (int32_t)j;
    }
    return off[nrows];
}

/* Same set through a uniform cell grid (cell edge = delta), an independent
 * second route used for large inputs.  Each row is sorted ascending. */
typedef struct {
    double lo[3];
    double h;
    int64_t dim[3];
    int64_t* start; /* ncell+1 */
    int64_t* items; /* node ids grouped by cell, ascending inside a cell */
} or_grid;

static int64_t cell_coord(double v, double lo, double h, int64_t dim)
{
    int64_t c = (int64_t)floor((v - lo) / h);
    if (c < 0) c = 0;
    if (c >= dim) c = dim - 1;
    return c;
}

static void grid_build(or_grid* g, const double* x, int64_t n, double delta)
{
    double hi[3];
    for (int a = 0; a < 3; ++a) { g->lo[a] = x[a]; hi[a] = x[a]; }
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            if (x[3 * i + a] < g->lo[a]) g->lo[a] = x[3 * i + a];
            if (x[3 * i + a] > hi[a]) hi[a] = x[3 * i + a];
        }
    g->h = delta;
    for (int a = 0; a < 3; ++a) g->dim[a] = (int64_t)floor((hi[a] - g->lo[a]) / delta) + 1;
    int64_t ncell = g->dim[0] * g->dim[1] * g->dim[2];
    g->start = (int64_t*)calloc((size_t)ncell + 1, sizeof(int64_t));
    g->items = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t* cell = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t c0 = cell_coord(x[3 * i], g->lo[0], g->h, g->dim[0]);
        int64_t c1 = cell_coord(x[3 * i + 1], g->lo[1], g->h, g->dim[1]);
        int64_t c2 = cell_coord(x[3 * i + 2], g->lo[2], g->h, g->dim[2]);
        cell[i] = (c0 * g->dim[1] + c1) * g->dim[2] + c2;
        g->start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) g->start[c + 1] += g->start[c];
    int64_t* fill = (int64_t*)malloc((size_t)ncell * sizeof(int64_t) + 8);
    memcpy(fill, g->start, (size_t)ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) g->items[fill[cell[i]]++] = i; /* ascending i */
    free(fill);
    free(cell);
}

static int cmp_i32(const void* a, const void* b)
{
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Visit the candidates of node i in the 27 surrounding cells. */
static int64_t grid_row(const or_grid* g, const double* x, int64_t i, double d2, int32_t* out)
{
    int64_t c[3];
    for (int a = 0; a < 3; ++a) c[a] = cell_coord(x[3 * i + a], g->lo[a], g->h, g->dim[a]);
    int64_t cnt = 0;
    for (int64_t a = c[0] - 1; a <= c[0] + 1; ++a) {
        if (a < 0 || a >= g->dim[0]) continue;
        for (int64_t b = c[1] - 1; b <= c[1] + 1; ++b) {
            if (b < 0 || b >= g->dim[1]) continue;
            for (int64_t d = c[2] - 1; d <= c[2] + 1; ++d) {
                if (d < 0 || d >= g->dim[2]) continue;
                int64_t cell = (a * g->dim[1] + b) * g->dim[2] + d;
                for (int64_t p = g->start[cell]; p < g->start[cell + 1]; ++p) {
                    int64_t j = g->items[p];
                    if (j != i && dist2(x + 3 * i, x + 3 * j) <= d2) {
                        if (out) out[cnt] = (int32_t)j;
                        ++cnt;
                    }
                }
            }
        }
    }
    if (out) qsort(out, (size_t)cnt, sizeof(int32_t), cmp_i32);
    return cnt;
}

int64_t or_family_cells(const double* x, int64_t n, double delta,
                        const int64_t* rows, int64_t nrows,
                        int64_t* off, int32_t* idx)
{
    or_grid g;
    grid_build(&g, x, n, delta);
    double d2 = delta * delta;
    if (idx == NULL) {
        int64_t* cnt = (int64_t*)malloc((size_t)(nrows > 0 ? nrows : 1) * sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t r = 0; r < nrows; ++r)
            cnt[r] = grid_row(&g, x, rows ? rows[r] : r, d2, NULL);
        off[0] = 0;
        for (int64_t r = 0; r < nrows; ++r) off[r + 1] = off[r] + cnt[r];
        free(cnt);
    } else {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t r = 0; r < nrows; ++r)
            grid_row(&g, x, rows ? rows[r] : r, d2, idx + off[r]);
    }
    free(g.start);
    free(g.items);
    return off[nrows];
}

/* ------------------------------------------------------------------ */
/* Initial notch (Section 6): the bond x_i -> x_j is absent when its segment
 * crosses the plane x[axis] = pos at a point inside the rectangle
 * lo_a <= x[a] <= hi_a, lo_b <= x[b] <= hi_b ((a, b) = other axes, ascending).
 * cut = {axis, pos, lo_a, hi_a, lo_b, hi_b}. */
int or_cut_crosses(const double* xi, const double* xj, const double* cut)
{
    int ax = (int)cut[0];
    double pos = cut[1];
    double di = xi[ax] - pos, dj = xj[ax] - pos;
    if (!(di * dj < 0.0)) return 0;
    double t = di / (di - dj);
    int a = (ax == 0) ? 1 : 0;
    int b = (ax == 2) ? 1 : 2;
    double pa = xi[a] + t * (xj[a] - xi[a]);
    double pb = xi[b] + t * (xj[b] - xi[b]);
    return pa >= cut[2] && pa <= cut[3] && pb >= cut[4] && pb <= cut[5];
}

/* keep[k] = 0 for every bond of the CSR family that crosses any cut, else 1. */
void or_apply_cuts(const double* x, const int64_t* rows, int64_t nrows,
                   const int64_t* off, const int32_t* idx,
                   const double* cuts, int64_t ncuts, uint8_t* keep)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows ? rows[r] : r;
        for (int64_t k = off[r]; k < off[r + 1]; ++k) {
            int64_t j = idx[k];
            uint8_t ok = 1;
            for (int64_t c = 0; c < ncuts && ok; ++c)
                if (or_cut_crosses(x + 3 * i, x + 3 * j, cuts + 6 * c)) ok = 0;
            keep[k] = ok;
        }
    }
}

/* ------------------------------------------------------------------ */
typedef struct {
    int64_t n;               /* number of nodes */
    const double* x;         /* 3n reference coordinates */
    const double* vol;       /* n nodal volumes */
    const int64_t* rows;     /* nrows node ids the family rows belong to, or NULL = 0..n-1 */
    int64_t nrows;
    const int64_t* off;      /* nrows+1 CSR offsets of the family (after notch removal) */
    const int32_t* idx;      /* neighbour ids, ascending within each row */
    double c;                /* micromodulus when c_bond == NULL */
    const double* c_bond;    /* per family entry, or NULL */
    double sc;               /* critical stretch when sc_mode == 0 */
    int32_t sc_mode;         /* 0 constant, 1 per-bond U[sc_lo, sc_hi) draw */
    int32_t pad0;
    uint64_t sc_seed;
    double sc_lo, sc_hi;
    const uint8_t* no_fail;  /* n flags or NULL: bonds touching such a node never break */
    const uint8_t* bc_type;  /* 3n: 1 = displacement-controlled component */
    const double* bc_disp;   /* 3n: prescribed displacement per unit scale */
    const double* bc_force;  /* 3n body-force density per unit load, or NULL */
    double disp_rate;        /* displacement scale rate (see or_scale below) */
    double load;             /* body-force scale */
    double dt, damping, density;
    int64_t ramp_steps;      /* 0: scale(k) = disp_rate k; T > 0: smooth start over T steps */
    double kr;               /* >= 1: bilinear softening with s_0 = s_c / kr; 0: PMB */
    double* kappa;           /* kr >= 1: largest stretch each family entry has reached */
    int32_t model;           /* 0 bond-based PMB; 1 ordinary state-based (linear solid) */
    int32_t pad1;
    double K, G;             /* model 1: bulk and shear modulus */
    double* wvol;            /* model 1: weighted volume m_i per node (or_osb_weighted_volume) */
    double* theta;           /* model 1: dilation per node, scratch of the step */
    double k1;               /* > 1: trilinear softening with the kink at s_1 = k1 s_0 */
    double beta;             /* trilinear: force at the kink / force at s_0 */
} or_model;

/* Bilinear bond law (Section 6, Example 3: the damage model of Gerstle et al.,
 * with s_0 the linear elastic limit and k_r = s_c / s_0): the force rises as
 * c s up to s_0, then falls linearly to zero at s_c.  The bond remembers the
 * largest stretch kappa it has reached, and below the envelope it unloads
 * towards the origin; its integrity is
 *   mu(kappa) = 1                                   kappa <= s_0
 *             = s_0 (s_c - kappa) / (kappa (s_c - s_0))   s_0 < kappa < s_c
 *             = 0 (broken, irreversibly)             kappa >= s_c
 * and the force is c s mu(kappa) V_j y/|y|.  kr = 1 (s_0 = s_c) is the PMB law
 * again, with the history kept. */
static double soft_mu(const or_model* m, double kappa, double s0, double sc)
{
    if (kappa <= s0) return 1.0;
    if (kappa >= sc) return 0.0;
    if (m->k1 > 1.0) {
        /* trilinear (Section 6, Example 2, after Yang et al.): the force falls
         * linearly from c s_0 at s_0 to beta c s_0 at the kink s_1, then to 0 at
         * s_c; mu = envelope / (c kappa) */
        double s1 = m->k1 * s0;
        if (kappa <= s1)
            return s0 * ((1.0 - m->beta) * (s1 - kappa) / (s1 - s0) + m->beta) / kappa;
        return s0 * m->beta * (sc - kappa) / ((sc - s1) * kappa);
    }
    return s0 * (sc - kappa) / (kappa * (sc - s0));
}

/* Displacement scale after step k.  Linear, rate * k, or with a smooth start
 * (Sections 5-6: a fifth-order polynomial displacement-time curve, so that the
 * loaded nodes start with zero acceleration and reach the steady rate with zero
 * acceleration): over the first T steps rate * T * P(k/T) with
 *   P(tau) = tau^4 - (3/5) tau^5,
 * whose value and first three derivatives vanish at 0, with P'(1) = 1,
 * P''(1) = 0 and P(1) = 2/5; afterwards the line rate * (k - 3T/5) that
 * continues it. */
double or_scale(double rate, int64_t ramp_steps, int64_t k)
{
    if (ramp_steps <= 0) return rate * (double)k;
    double T = (double)ramp_steps;
    if (k >= ramp_steps) return rate * ((double)k - 0.6 * T);
    double tau = (double)k / T;
    return rate * T * (tau * tau * tau * tau - 0.6 * tau * tau * tau * tau * tau);
}

static double bond_sc(const or_model* m, int64_t i, int64_t j)
{
    if (m->sc_mode == 1) return or_sc_bond(m->sc_seed, m->sc_lo, m->sc_hi, i, j);
    return m->sc;
}

/* Internal force density of row r (Eq. (10) sum with beta = 1) and the bond
 * updates of Algorithm bond_index: for every intact bond compute the stretch
 * (Eq. (4)); if s >= s_c the bond breaks for good (Eq. (6)) and adds nothing;
 * else it adds c s V_j (xi+eta)/|xi+eta| (Eq. (5)). */
static void row_force(const or_model* m, int64_t r, const double* u, uint8_t* mu,
                      double* margin, double F[3])
{
    int64_t i = m->rows ? m->rows[r] : r;
    F[0] = F[1] = F[2] = 0.0;
    for (int64_t k = m->off[r]; k < m->off[r + 1]; ++k) {
        if (!mu[k]) continue;
        int64_t j = m->idx[k];
        double xi[3], eta[3], y[3];
        for (int a = 0; a < 3; ++a) {
            xi[a] = m->x[3 * j + a] - m->x[3 * i + a];
            eta[a] = u[3 * j + a] - u[3 * i + a];
            y[a] = xi[a] + eta[a];
        }
        double L = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
        double rr = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
        double s = (rr - L) / L;
        double sc = bond_sc(m, i, j);
        if (margin) {
            double d = fabs(s - sc);
            if (d < margin[k]) margin[k] = d;
        }
        int nofail = m->no_fail && (m->no_fail[i] || m->no_fail[j]);
        double kap = s;
        if (m->kr >= 1.0) {
            kap = m->kappa[k] > s ? m->kappa[k] : s;
            m->kappa[k] = kap;
        }
        if (kap >= sc && !nofail) {
            mu[k] = 0;
            continue;
        }
        double cij = m->c_bond ? m->c_bond[k] : m->c;
        double f = cij * s * m->vol[j] / rr;
        if (m->kr >= 1.0) f = cij * s * soft_mu(m, kap, sc / m->kr, sc) * m->vol[j] / rr;
        for (int a = 0; a < 3; ++a) F[a] += f * y[a];
    }
    if (m->bc_force)
        for (int a = 0; a < 3; ++a) F[a] += m->load * m->bc_force[3 * i + a];
}

/* One damped Euler-Cromer step from (u, v) at step index `step` (t = step*dt)
 * for the rows of the model.  mu (per family entry) is updated in place;
 * margin (per family entry, or NULL) keeps min |s - s_c| over intact bonds.
 * Outputs are per row: u_out, v_out (3 per row) and, if F_out != NULL, the
 * force density F_i of Eq. (11) before integration. */
/* ------------------------------------------------------------------ */
/* Ordinary state-based peridynamics (Section "State-based Peridynamics": two
 * loops per step, a nodal dilation and then the nodal force), with the linear
 * peridynamic solid of Silling et al. (2007) as the material and a constant
 * influence function omega = 1:
 *   m_i     = sum_j |xi_ij|^2 V_j                      (weighted volume, reference)
 *   e_ij    = |y_ij| - |xi_ij|                         (bond extension)
 *   theta_i = (3 / m_i) sum_j mu_ij |xi_ij| e_ij V_j    (dilation)
 *   t_ij    = (3 K theta_i / m_i) |xi_ij| + (15 G / m_i) (e_ij - theta_i |xi_ij| / 3)
 *   F_i     = sum_j mu_ij (t_ij + t_ji) y_ij / |y_ij| V_j
 * Bonds break in the dilation loop with the rule of Eq. (6) (s = e / |xi|), so
 * a bond breaking in a step contributes to neither loop.  All nodes are rows. */
void or_osb_weighted_volume(const or_model* m, double* out)
{
    for (int64_t i = 0; i < m->n; ++i) {
        double acc = 0.0;
        for (int64_t k = m->off[i]; k < m->off[i + 1]; ++k)
            acc += dist2(m->x + 3 * i, m->x + 3 * m->idx[k]) * m->vol[m->idx[k]];
        out[i] = acc;
    }
}

static void bond_geom(const or_model* m, int64_t i, int64_t j, const double* u, double* L,
                      double* rr, double y[3])
{
    double xi[3];
    for (int a = 0; a < 3; ++a) {
        xi[a] = m->x[3 * j + a] - m->x[3 * i + a];
        y[a] = xi[a] + u[3 * j + a] - u[3 * i + a];
    }
    *L = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    *rr = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
}

/* dilation of every node (first loop); breaks bonds if `breaking` */
static void osb_dilation(const or_model* m, const double* u, uint8_t* mu, double* margin,
                         int breaking)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < m->n; ++i) {
        double acc = 0.0;
        for (int64_t k = m->off[i]; k < m->off[i + 1]; ++k) {
            if (!mu[k]) continue;
            int64_t j = m->idx[k];
            double L, rr, y[3];
            bond_geom(m, i, j, u, &L, &rr, y);
            if (breaking) {
                double s = (rr - L) / L;
                double sc = bond_sc(m, i, j);
                if (margin) {
                    double d = fabs(s - sc);
                    if (d < margin[k]) margin[k] = d;
                }
                int nofail = m->no_fail && (m->no_fail[i] || m->no_fail[j]);
                if (s >= sc && !nofail) {
                    mu[k] = 0;
                    continue;
                }
            }
            acc += L * (rr - L) * m->vol[j];
        }
        m->theta[i] = m->wvol[i] > 0.0 ? 3.0 * acc / m->wvol[i] : 0.0;
    }
}

/* force density of node i (second loop) from the dilations */
static void osb_force(const or_model* m, int64_t i, const double* u, const uint8_t* mu,
                      double F[3])
{
    F[0] = F[1] = F[2] = 0.0;
    for (int64_t k = m->off[i]; k < m->off[i + 1]; ++k) {
        if (!mu[k]) continue;
        int64_t j = m->idx[k];
        double L, rr, y[3];
        bond_geom(m, i, j, u, &L, &rr, y);
        double e = rr - L;
        double ti = 3.0 * m->K * m->theta[i] / m->wvol[i] * L +
                    15.0 * m->G / m->wvol[i] * (e - m->theta[i] * L / 3.0);
        double tj = 3.0 * m->K * m->theta[j] / m->wvol[j] * L +
                    15.0 * m->G / m->wvol[j] * (e - m->theta[j] * L / 3.0);
        double f = (ti + tj) * m->vol[j] / rr;
        for (int a = 0; a < 3; ++a) F[a] += f * y[a];
    }
    if (m->bc_force)
        for (int a = 0; a < 3; ++a) F[a] += m->load * m->bc_force[3 * i + a];
}

/* strain energy density of the linear solid:
 * W_i = K theta_i^2 / 2 + (15 G / (2 m_i)) sum_j mu_ij (e_ij - theta_i |xi_ij| / 3)^2 V_j */
static void osb_energy(const or_model* m, const double* u, const uint8_t* mu, double* W)
{
    osb_dilation(m, u, (uint8_t*)mu, NULL, 0);
    for (int64_t i = 0; i < m->n; ++i) {
        double acc = 0.0;
        for (int64_t k = m->off[i]; k < m->off[i + 1]; ++k) {
            if (!mu[k]) continue;
            int64_t j = m->idx[k];
            double L, rr, y[3];
            bond_geom(m, i, j, u, &L, &rr, y);
            double ed = (rr - L) - m->theta[i] * L / 3.0;
            acc += ed * ed * m->vol[j];
        }
        W[i] = 0.5 * m->K * m->theta[i] * m->theta[i] +
               (m->wvol[i] > 0.0 ? 7.5 * m->G / m->wvol[i] * acc : 0.0);
    }
}

void or_step(const or_model* m, int64_t step, const double* u, const double* v,
             uint8_t* mu, double* margin, double* u_out, double* v_out, double* F_out)
{
    if (m->model == 1) osb_dilation(m, u, mu, margin, 1);
    double a_damp = m->damping, rho = m->density, dt = m->dt;
    double s_now = or_scale(m->disp_rate, m->ramp_steps, step);
    double s_next = or_scale(m->disp_rate, m->ramp_steps, step + 1);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t r = 0; r < m->nrows; ++r) {
        int64_t i = m->rows ? m->rows[r] : r;
        double F[3];
        if (m->model == 1)
            osb_force(m, i, u, mu, F);
        else
            row_force(m, r, u, mu, margin, F);
        for (int a = 0; a < 3; ++a) {
            double vi = v[3 * i + a];
            double vn = vi + dt * (F[a] - a_damp * vi) / rho;
            double un = u[3 * i + a] + dt * vn;
            if (m->bc_type[3 * i + a] == 1) {
                double g = m->bc_disp[3 * i + a];
                un = g * s_next;
                vn = g * (s_next - s_now) / dt;
            }
            u_out[3 * r + a] = un;
            v_out[3 * r + a] = vn;
            if (F_out) F_out[3 * r + a] = F[a];
        }
    }
}

/* Run `nsteps` steps over all nodes (rows must be NULL): u, v in/out, mu in/out. */
void or_run(const or_model* m, int64_t first_step, int64_t nsteps, double* u, double* v,
            uint8_t* mu, double* margin)
{
    int64_t n3 = 3 * m->n;
    double* u2 = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    double* v2 = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    for (int64_t k = 0; k < nsteps; ++k) {
        or_step(m, first_step + k, u, v, mu, margin, u2, v2, NULL);
        memcpy(u, u2, (size_t)n3 * sizeof(double));
        memcpy(v, v2, (size_t)n3 * sizeof(double));
    }
    free(u2);
    free(v2);
}

/* Damped velocity-Verlet (Section 3.6, "Time integration"; the velocity-
 * dependent damping force after Groot & Warren 1997 with lambda = 1/2).  State
 * (u^n, v^n, a^n) at step n; one step, for free components:
 *   u^{n+1} = u^n + dt v^n + (dt^2/2) a^n
 *   vt      = v^n + (dt/2) a^n                        (half-step velocity)
 *   a^{n+1} = (F(u^{n+1}) - eta vt) / rho              (F at the new positions,
 *                                                        bonds breaking there first)
 *   v^{n+1} = v^n + (dt/2) (a^n + a^{n+1})
 * Displacement-controlled components: u^{n+1} = g scale(n+1),
 * v^{n+1} = g (scale(n+1) - scale(n)) / dt, a^{n+1} = 0.
 * With init != 0 the acceleration of the initial state is formed first,
 * a^0 = (F(u^0) - eta v^0) / rho (bonds past s_c at u^0 break).  All nodes are
 * rows.  u, v, a, mu in/out; margin (or NULL) keeps min |s - s_c| per entry. */
static void vv_accel(const or_model* m, const double* u, const double* vt, uint8_t* mu,
                     double* margin, double* acc)
{
    /* the state-based model: its first loop (dilations, bonds past s_c break)
     * before the forces, as in or_step */
    if (m->model == 1) osb_dilation(m, u, mu, margin, 1);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < m->n; ++i) {
        double F[3];
        if (m->model == 1)
            osb_force(m, i, u, mu, F);
        else
            row_force(m, i, u, mu, margin, F);
        for (int a = 0; a < 3; ++a)
            acc[3 * i + a] = m->bc_type[3 * i + a] == 1
                                 ? 0.0
                                 : (F[a] - m->damping * vt[3 * i + a]) / m->density;
    }
}

void or_run_vv(const or_model* m, int64_t first_step, int64_t nsteps, int init, double* u,
               double* v, double* acc, uint8_t* mu, double* margin)
{
    int64_t n3 = 3 * m->n;
    double dt = m->dt;
    double* vt = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    double* an = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    if (init) vv_accel(m, u, v, mu, margin, acc);
    for (int64_t k = 0; k < nsteps; ++k) {
        int64_t step = first_step + k;
        double s_now = or_scale(m->disp_rate, m->ramp_steps, step);
        double s_next = or_scale(m->disp_rate, m->ramp_steps, step + 1);
        for (int64_t e = 0; e < n3; ++e) {
            if (m->bc_type[e] == 1) {
                u[e] = m->bc_disp[e] * s_next;
                vt[e] = 0.0;
            } else {
                u[e] = u[e] + dt * v[e] + 0.5 * dt * dt * acc[e];
                vt[e] = v[e] + 0.5 * dt * acc[e];
            }
        }
        vv_accel(m, u, vt, mu, margin, an);
        for (int64_t e = 0; e < n3; ++e) {
            if (m->bc_type[e] == 1)
                v[e] = m->bc_disp[e] * (s_next - s_now) / dt;
            else
                v[e] = v[e] + 0.5 * dt * (acc[e] + an[e]);
            acc[e] = an[e];
        }
    }
    free(vt);
    free(an);
}

/* Eq. (8) with volume weights: phi_i = 1 - sum_j mu_ij V_j / sum_j V_j over the
 * family of i (after the initial notch removal). */
void or_damage(const or_model* m, const uint8_t* mu, double* phi)
{
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m->nrows; ++r) {
        double num = 0.0, den = 0.0;
        int64_t i = m->rows ? m->rows[r] : r;
        for (int64_t k = m->off[r]; k < m->off[r + 1]; ++k) {
            double vj = m->vol[m->idx[k]];
            den += vj;
            if (!mu[k]) continue;
            if (m->kr >= 1.0) {
                /* Eq. (8) with the bond's integrity mu(kappa) in [0, 1] */
                double sc = bond_sc(m, i, m->idx[k]);
                num += soft_mu(m, m->kappa[k], sc / m->kr, sc) * vj;
            } else {
                num += vj;
            }
        }
        phi[r] = den > 0.0 ? 1.0 - num / den : 0.0;
    }
}

/* Elastic energy density of each row: W_i = 1/2 sum_j mu_ij w(eta, xi) V_j with
 * the micropotential of Eq. (4) read as w = c s^2 |xi| / 2 (the factor 1/2
 * shares each bond's energy between its two end nodes). */
void or_energy_density(const or_model* m, const double* u, const uint8_t* mu, double* W)
{
    if (m->model == 1) {
        osb_energy(m, u, mu, W);
        return;
    }
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < m->nrows; ++r) {
        int64_t i = m->rows ? m->rows[r] : r;
        double acc = 0.0;
        for (int64_t k = m->off[r]; k < m->off[r + 1]; ++k) {
            if (!mu[k]) continue;
            int64_t j = m->idx[k];
            double xi[3], y[3];
            for (int a = 0; a < 3; ++a) {
                xi[a] = m->x[3 * j + a] - m->x[3 * i + a];
                y[a] = xi[a] + u[3 * j + a] - u[3 * i + a];
            }
            double L = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
            double rr = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
            double s = (rr - L) / L;
            double cij = m->c_bond ? m->c_bond[k] : m->c;
            acc += 0.5 * (0.5 * cij * s * s * L) * m->vol[j];
        }
        W[r] = acc;
    }
}

/* ------------------------------------------------------------------ */
/* Stiffness corrections as per-bond factors that multiply the constant
 * micromodulus c of Eq. (5), one per family entry (Section 2.2, micromodulus
 * functions; "Surface correction factors"):
 *   bit 0, conical micromodulus c(|xi|) = c1 (1 - |xi|/delta): the strain
 *     energy density under uniform dilation s = eps,
 *       W = (eps^2 / 4) int_0^delta c(r) r 4 pi r^2 dr = (eps^2 / 4) c1 pi delta^4 / 5,
 *     equated to (9/2) K eps^2 gives c1 = 90 K / (pi delta^4) = 5 c, so the
 *     factor is 5 (1 - |xi| / delta);
 *   bit 1, volume (surface) correction lambda_ij = 2 V0 / (V_i + V_j) with V_i
 *     the family volume sum_{j in H_i} V_j of node i (family as given, i.e.
 *     after the initial notch removal) and V0 the family volume of a node in
 *     the bulk (an input).
 *   bit 2, partial volume (Section 2.3, beta_ij of the discrete equation of
 *     motion): the fraction of node j's cell inside the horizon, taken as the
 *     linear rule beta = (delta + dx/2 - |xi|) / dx clipped to [0, 1], dx = dx_pv
 *     the lattice spacing (a family built with horizon delta + dx/2 gives the
 *     cells straddling the horizon their outer part too);
 * With several bits the factors multiply.  All nodes are rows. */
static double partial_volume(double L, double delta, double dx)
{
    double b = (delta + 0.5 * dx - L) / dx;
    return b < 0.0 ? 0.0 : (b > 1.0 ? 1.0 : b);
}

void or_stiffness_factors2(const double* x, const double* vol, int64_t n, double delta,
                           const int64_t* off, const int32_t* idx, int flags, double v0,
                           double dx_pv, double* out);

void or_stiffness_factors(const double* x, const double* vol, int64_t n, double delta,
                          const int64_t* off, const int32_t* idx, int flags, double v0,
                          double* out)
{
    or_stiffness_factors2(x, vol, n, delta, off, idx, flags, v0, 0.0, out);
}

void or_stiffness_factors2(const double* x, const double* vol, int64_t n, double delta,
                           const int64_t* off, const int32_t* idx, int flags, double v0,
                           double dx_pv, double* out)
{
    double* fv = NULL;
    if (flags & 2) {
        fv = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
        for (int64_t i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int64_t k = off[i]; k < off[i + 1]; ++k) acc += vol[idx[k]];
            fv[i] = acc;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = off[i]; k < off[i + 1]; ++k) {
            int64_t j = idx[k];
            double f = 1.0;
            if (flags & 1) {
                double L = sqrt(dist2(x + 3 * i, x + 3 * j));
                f *= 5.0 * (1.0 - L / delta);
            }
            if (flags & 2) f *= 2.0 * v0 / (fv[i] + fv[j]);
            if (flags & 4) f *= partial_volume(sqrt(dist2(x + 3 * i, x + 3 * j)), delta, dx_pv);
            out[k] = f;
        }
    free(fv);
}

/* ------------------------------------------------------------------ */
/* Reverse mode of the damped Euler-Cromer recurrence with the bond flags mu
 * frozen (no bond changes state during the run).  Forward, for free components:
 *   F^n = sum_j c_ij mu_ij s_ij V_j y_ij/|y_ij| + load * force_i      (Eqs. 5, 10)
 *   v^{n+1} = v^n + dt (F^n - eta v^n) / rho,  u^{n+1} = u^n + dt v^{n+1}
 * and controlled components are overwritten by the prescribed ramp.  With
 * ubar, vbar the adjoints of u^{n+1}, v^{n+1} (controlled components zeroed):
 *   w = vbar + dt ubar
 *   ubar^n = ubar + (dt/rho) (J^T w),  vbar^n = (1 - dt eta/rho) w
 *   (J^T w)_m = sum_{j in H_m} c_mj mu_mj K_mj (V_m w_j - V_j w_m),
 *   K = (1/L - 1/r) I + y y^T / r^3   (L = |xi|, r = |y|; d/dy of s y/|y|)
 *   dL/dc[m->j] += (dt/rho) mu s V_j (y/r).w_m   (c of the directed entry m->j,
 *              which only enters F_m; an undirected bond's sensitivity is the
 *              sum over its two directed entries)
 *   dL/dload += (dt/rho) sum_m force_m . w_m
 * All nodes must be rows (m->rows == NULL).  Stores every u^n (small cases). */
void or_adjoint(const or_model* m, int64_t first_step, int64_t nsteps, const double* u0,
                const double* v0, const uint8_t* mu, const double* dLdu, const double* dLdv,
                double* dLdc, double* dLdload, double* dLdu0, double* dLdv0)
{
    const int64_t n = m->n, n3 = 3 * n;
    double* U = (double*)malloc((size_t)(nsteps + 1) * n3 * sizeof(double) + 8);
    double* v = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    double* u2 = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    double* v2 = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    uint8_t* muc = (uint8_t*)malloc((size_t)(m->off[n] > 0 ? m->off[n] : 1));
    memcpy(U, u0, (size_t)n3 * sizeof(double));
    memcpy(v, v0, (size_t)n3 * sizeof(double));
    for (int64_t k = 0; k < nsteps; ++k) {
        memcpy(muc, mu, (size_t)m->off[n]);
        or_step(m, first_step + k, U + k * n3, v, muc, NULL, u2, v2, NULL);
        memcpy(U + (k + 1) * n3, u2, (size_t)n3 * sizeof(double));
        memcpy(v, v2, (size_t)n3 * sizeof(double));
    }
    double* ub = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    double* vb = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    double* w = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    memcpy(ub, dLdu, (size_t)n3 * sizeof(double));
    for (int64_t e = 0; e < n3; ++e) vb[e] = dLdv ? dLdv[e] : 0.0;
    for (int64_t k = 0; k < m->off[n]; ++k) dLdc[k] = 0.0;
    double gload = 0.0;
    const double dr = m->dt / m->density, a = 1.0 - m->dt * m->damping / m->density;
    for (int64_t k = nsteps - 1; k >= 0; --k) {
        const double* u = U + k * n3; /* u^k: the state the step k -> k+1 reads */
        for (int64_t e = 0; e < n3; ++e) {
            if (m->bc_type[e] == 1) {
                ub[e] = 0.0;
                vb[e] = 0.0;
            }
            w[e] = vb[e] + m->dt * ub[e];
        }
        if (m->bc_force)
            for (int64_t e = 0; e < n3; ++e) gload += dr * m->bc_force[e] * w[e];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double acc[3] = {0.0, 0.0, 0.0};
            for (int64_t q = m->off[i]; q < m->off[i + 1]; ++q) {
                if (!mu[q]) continue;
                const int64_t j = m->idx[q];
                double xi[3], y[3], d[3];
                for (int c = 0; c < 3; ++c) {
                    xi[c] = m->x[3 * j + c] - m->x[3 * i + c];
                    y[c] = xi[c] + u[3 * j + c] - u[3 * i + c];
                    d[c] = m->vol[i] * w[3 * j + c] - m->vol[j] * w[3 * i + c];
                }
                const double L = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
                const double r = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
                const double s = (r - L) / L;
                const double yd = y[0] * d[0] + y[1] * d[1] + y[2] * d[2];
                const double cij = m->c_bond ? m->c_bond[q] : m->c;
                for (int c = 0; c < 3; ++c)
                    acc[c] += cij * ((1.0 / L - 1.0 / r) * d[c] + y[c] * yd / (r * r * r));
                const double yw = y[0] * w[3 * i] + y[1] * w[3 * i + 1] + y[2] * w[3 * i + 2];
                dLdc[q] += dr * s * m->vol[j] * yw / r;
            }
            for (int c = 0; c < 3; ++c) {
                u2[3 * i + c] = ub[3 * i + c] + dr * acc[c];
                v2[3 * i + c] = a * w[3 * i + c];
            }
        }
        memcpy(ub, u2, (size_t)n3 * sizeof(double));
        memcpy(vb, v2, (size_t)n3 * sizeof(double));
    }
    if (dLdload) *dLdload = gload;
    if (dLdu0) memcpy(dLdu0, ub, (size_t)n3 * sizeof(double));
    if (dLdv0) memcpy(dLdv0, vb, (size_t)n3 * sizeof(double));
    free(U); free(v); free(u2); free(v2); free(muc); free(ub); free(vb); free(w);
}

/* out += scale (J^T w) at u, with J = dF/du of the pairwise force density
 * (frozen flags mu), and the matching stiffness and load sensitivities:
 *   dLdc[m->j] += scale mu s V_j (y/r).w_m,   *gload += scale sum_m force_m . w_m
 * (the terms of or_adjoint's reverse step, with w given). */
static void jt_accumulate(const or_model* m, const double* u, const double* w,
                          const uint8_t* mu, double scale, double* out, double* dLdc,
                          double* gload)
{
    const int64_t n = m->n;
    if (m->bc_force)
        for (int64_t e = 0; e < 3 * n; ++e) *gload += scale * m->bc_force[e] * w[e];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double acc[3] = {0.0, 0.0, 0.0};
        for (int64_t q = m->off[i]; q < m->off[i + 1]; ++q) {
            if (!mu[q]) continue;
            const int64_t j = m->idx[q];
            double xi[3], y[3], d[3];
            for (int c = 0; c < 3; ++c) {
                xi[c] = m->x[3 * j + c] - m->x[3 * i + c];
                y[c] = xi[c] + u[3 * j + c] - u[3 * i + c];
                d[c] = m->vol[i] * w[3 * j + c] - m->vol[j] * w[3 * i + c];
            }
            const double L = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
            const double r = sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]);
            const double s = (r - L) / L;
            const double yd = y[0] * d[0] + y[1] * d[1] + y[2] * d[2];
            const double cij = m->c_bond ? m->c_bond[q] : m->c;
            for (int c = 0; c < 3; ++c)
                acc[c] += cij * ((1.0 / L - 1.0 / r) * d[c] + y[c] * yd / (r * r * r));
            const double yw = y[0] * w[3 * i] + y[1] * w[3 * i + 1] + y[2] * w[3 * i + 2];
            dLdc[q] += scale * s * m->vol[j] * yw / r;
        }
        for (int c = 0; c < 3; ++c) out[3 * i + c] += scale * acc[c];
    }
}

/* Reverse mode of the damped velocity-Verlet run of or_run_vv started with
 * init = 1 (a^0 formed from the initial state), bond flags frozen (mu), for a
 * loss L(u^N, v^N).  Each assignment of the forward step, in its order
 *   a^0     = P (F(u^0) - eta v^0) / rho
 *   u^{n+1} = u^n + dt v^n + dt^2/2 a^n          (free components)
 *   vt      = v^n + dt/2 a^n                      (free components, else 0)
 *   a^{n+1} = P (F(u^{n+1}) - eta vt) / rho
 *   v^{n+1} = v^n + dt/2 (a^n + a^{n+1})          (free components)
 * (P keeps the free components; controlled ones follow the prescribed ramp and
 * do not depend on the state), is reversed in the opposite order with the
 * adjoints ubar, vbar, abar of u, v, a.  F = F_int + load b, and
 * d(J^T)/dc, db as in or_adjoint.  Stores every u^n (small cases). */
void or_adjoint_vv(const or_model* m, int64_t first_step, int64_t nsteps, const double* u0,
                   const double* v0, const uint8_t* mu, const double* dLdu, const double* dLdv,
                   double* dLdc, double* dLdload, double* dLdu0, double* dLdv0)
{
    const int64_t n = m->n, n3 = 3 * n;
    const double dt = m->dt, rho = m->density, eta = m->damping;
    double* U = (double*)malloc((size_t)(nsteps + 1) * n3 * sizeof(double) + 8);
    double* v = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    double* a = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    uint8_t* muc = (uint8_t*)malloc((size_t)(m->off[n] > 0 ? m->off[n] : 1));
    memcpy(U, u0, (size_t)n3 * sizeof(double));
    memcpy(v, v0, (size_t)n3 * sizeof(double));
    memcpy(muc, mu, (size_t)(m->off[n] > 0 ? m->off[n] : 1));
    /* forward, keeping u^n; frozen flags: the run must not break a bond */
    or_run_vv(m, first_step, 0, 1, U, v, a, muc, NULL);
    for (int64_t k = 0; k < nsteps; ++k) {
        memcpy(U + (k + 1) * n3, U + k * n3, (size_t)n3 * sizeof(double));
        or_run_vv(m, first_step + k, 1, 0, U + (k + 1) * n3, v, a, muc, NULL);
    }
    double* ub = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    double* vb = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    double* ab = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    double* t = (double*)malloc((size_t)n3 * sizeof(double) + 8);
    memcpy(ub, dLdu, (size_t)n3 * sizeof(double));
    for (int64_t e = 0; e < n3; ++e) {
        vb[e] = dLdv ? dLdv[e] : 0.0;
        ab[e] = 0.0;
    }
    for (int64_t k = 0; k < m->off[n]; ++k) dLdc[k] = 0.0;
    double gload = 0.0;
    for (int64_t k = nsteps - 1; k >= 0; --k) {
        /* v^{k+1} = v^k + dt/2 (a^k + a^{k+1}) */
        for (int64_t e = 0; e < n3; ++e) {
            if (m->bc_type[e] == 1) vb[e] = 0.0;
            ab[e] += 0.5 * dt * vb[e];
        }
        /* a^{k+1} = P (F(u^{k+1}) - eta vt) / rho */
        for (int64_t e = 0; e < n3; ++e) t[e] = m->bc_type[e] == 1 ? 0.0 : ab[e];
        jt_accumulate(m, U + (k + 1) * n3, t, mu, 1.0 / rho, ub, dLdc, &gload);
        /* vt = v^k + dt/2 a^k, u^{k+1} = u^k + dt v^k + dt^2/2 a^k (free components) */
        for (int64_t e = 0; e < n3; ++e) {
            const double vtb = -eta / rho * t[e];
            const double up = m->bc_type[e] == 1 ? 0.0 : ub[e];
            const double vbk = vb[e] + vtb + dt * up;
            ab[e] = 0.5 * dt * vb[e] + 0.5 * dt * vtb + 0.5 * dt * dt * up;
            vb[e] = vbk;
            ub[e] = up;
        }
    }
    /* a^0 = P (F(u^0) - eta v^0) / rho */
    for (int64_t e = 0; e < n3; ++e) t[e] = m->bc_type[e] == 1 ? 0.0 : ab[e];
    jt_accumulate(m, U, t, mu, 1.0 / rho, ub, dLdc, &gload);
    for (int64_t e = 0; e < n3; ++e) vb[e] += -eta / rho * t[e];
    if (dLdload) *dLdload = gload;
    if (dLdu0) memcpy(dLdu0, ub, (size_t)n3 * sizeof(double));
    if (dLdv0) memcpy(dLdv0, vb, (size_t)n3 * sizeof(double));
    free(U); free(v); free(a); free(muc); free(ub); free(vb); free(ab); free(t);
}
