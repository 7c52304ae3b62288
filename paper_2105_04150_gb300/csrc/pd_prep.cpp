// Host-side model preparation: family search, initial notch removal, spatial
// node order, padded device layout, boundary-condition classes and the
// explicit stability bound.  Runs once per pd_create (the paper builds the
// neighbour list once per model, Section 3 "reduced overhead").
#include "pd_prep.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>

namespace pd {

namespace {

struct Grid {
    double lo[3];
    double h;
    int64_t dim[3];
    std::vector<int64_t> start;  // ncell + 1
    std::vector<int32_t> items;  // node ids grouped by cell, ascending in a cell
};

int64_t cell_of(double v, double lo, double h, int64_t dim)
{
    int64_t c = (int64_t)std::floor((v - lo) / h);
    return c < 0 ? 0 : (c >= dim ? dim - 1 : c);
}

bool build_grid(Grid& g, int64_t n, const double* x, double h)
{
    double hi[3];
    for (int a = 0; a < 3; ++a) g.lo[a] = hi[a] = x[a];
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            g.lo[a] = std::min(g.lo[a], x[3 * i + a]);
            hi[a] = std::max(hi[a], x[3 * i + a]);
        }
    g.h = h;
    double ncell = 1.0;
    for (int a = 0; a < 3; ++a) {
        g.dim[a] = (int64_t)std::floor((hi[a] - g.lo[a]) / h) + 1;
        ncell *= (double)g.dim[a];
    }
    if (ncell > 4.0e9) return false;
    const int64_t nc = g.dim[0] * g.dim[1] * g.dim[2];
    g.start.assign(nc + 1, 0);
    g.items.resize(n);
    std::vector<int64_t> cell(n);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t c0 = cell_of(x[3 * i], g.lo[0], h, g.dim[0]);
        const int64_t c1 = cell_of(x[3 * i + 1], g.lo[1], h, g.dim[1]);
        const int64_t c2 = cell_of(x[3 * i + 2], g.lo[2], h, g.dim[2]);
        cell[i] = (c0 * g.dim[1] + c1) * g.dim[2] + c2;
        g.start[cell[i] + 1]++;
    }
    for (int64_t c = 0; c < nc; ++c) g.start[c + 1] += g.start[c];
    std::vector<int64_t> fill(g.start.begin(), g.start.end() - 1);
    for (int64_t i = 0; i < n; ++i) g.items[fill[cell[i]]++] = (int32_t)i;
    return true;
}

// Members j != i with |x_j - x_i|^2 <= delta^2 (Eq. 9), in the 27 cells around i.
template <class Emit>
void scan_neighbours(const Grid& g, const double* x, int64_t i, double d2, Emit emit)
{
    int64_t c[3];
    for (int a = 0; a < 3; ++a) c[a] = cell_of(x[3 * i + a], g.lo[a], g.h, g.dim[a]);
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    for (int64_t a = std::max<int64_t>(c[0] - 1, 0); a <= std::min(c[0] + 1, g.dim[0] - 1); ++a)
        for (int64_t b = std::max<int64_t>(c[1] - 1, 0); b <= std::min(c[1] + 1, g.dim[1] - 1); ++b)
            for (int64_t e = std::max<int64_t>(c[2] - 1, 0); e <= std::min(c[2] + 1, g.dim[2] - 1);
                 ++e) {
                const int64_t cell = (a * g.dim[1] + b) * g.dim[2] + e;
                for (int64_t p = g.start[cell]; p < g.start[cell + 1]; ++p) {
                    const int32_t j = g.items[p];
                    if (j == i) continue;
                    const double dx = x[3 * j] - xi, dy = x[3 * j + 1] - yi, dz = x[3 * j + 2] - zi;
                    if (dx * dx + dy * dy + dz * dz <= d2) emit(j);
                }
            }
}

}  // namespace

std::string search_family(int64_t n, const double* x, double delta, std::vector<int64_t>& off,
                          std::vector<int32_t>& idx)
{
    Grid g;
    if (!build_grid(g, n, x, delta)) return "horizon too small for the extent of the body";
    const double d2 = delta * delta;
    off.assign(n + 1, 0);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        int64_t cnt = 0;
        scan_neighbours(g, x, i, d2, [&](int32_t) { ++cnt; });
        off[i + 1] = cnt;
    }
    for (int64_t i = 0; i < n; ++i) off[i + 1] += off[i];
    idx.resize(off[n]);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        int64_t p = off[i];
        scan_neighbours(g, x, i, d2, [&](int32_t j) { idx[p++] = j; });
        std::sort(idx.begin() + off[i], idx.begin() + off[i + 1]);
    }
    return "";
}

std::string check_family(int64_t n, const int64_t* off, const int32_t* idx)
{
    if (off[0] != 0) return "family offsets must start at 0";
    for (int64_t i = 0; i < n; ++i) {
        if (off[i + 1] < off[i]) return "family offsets must be non-decreasing";
        for (int64_t k = off[i]; k < off[i + 1]; ++k) {
            const int32_t j = idx[k];
            if (j < 0 || j >= n || j == i) return "family index out of range or self-bond";
            if (k > off[i] && idx[k - 1] >= j) return "family rows must be strictly ascending";
        }
    }
    // symmetry: j in H_i  <=>  i in H_j
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = off[i]; k < off[i + 1]; ++k) {
            const int32_t j = idx[k];
            if (!std::binary_search(idx + off[j], idx + off[j + 1], (int32_t)i))
                return "family must be symmetric";
        }
    return "";
}

// A bond x_i -> x_j is removed when its segment meets the plane
// x[axis] = pos strictly between its end points at a point of the rectangle.
static bool crosses(const double* xi, const double* xj, const double* cut)
{
    const int ax = (int)cut[0];
    const double a0 = xi[ax] - cut[1], a1 = xj[ax] - cut[1];
    if (!(a0 * a1 < 0.0)) return false;
    const double t = a0 / (a0 - a1);
    int o = 0;
    double pt[2];
    for (int a = 0; a < 3; ++a) {
        if (a == ax) continue;
        pt[o++] = xi[a] + t * (xj[a] - xi[a]);
    }
    return pt[0] >= cut[2] && pt[0] <= cut[3] && pt[1] >= cut[4] && pt[1] <= cut[5];
}

void apply_cuts(int64_t n, const double* x, const double* cuts, int32_t ncuts,
                std::vector<int64_t>& off, std::vector<int32_t>& idx)
{
    if (ncuts <= 0) return;
    std::vector<uint8_t> keep(idx.size(), 1);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = off[i]; k < off[i + 1]; ++k)
            for (int32_t c = 0; c < ncuts; ++c)
                if (crosses(x + 3 * i, x + 3 * (int64_t)idx[k], cuts + 6 * c)) {
                    keep[k] = 0;
                    break;
                }
    int64_t w = 0;
    std::vector<int64_t> noff(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = off[i]; k < off[i + 1]; ++k)
            if (keep[k]) idx[w++] = idx[k];
        noff[i + 1] = w;
    }
    idx.resize(w);
    off.swap(noff);
}

void spatial_order(int64_t n, const double* x, double delta, int reorder,
                   std::vector<int32_t>& perm, std::vector<int32_t>& inv)
{
    // reorder == 0 keeps the caller's order (a row-major lattice is already the
    // best order for the sliced layout: the 32 nodes of a slice are translates
    // of each other, so slot m of all of them points to the same offset and the
    // neighbour gathers are contiguous).  reorder == 1 sorts nodes by the cell
    // (edge = horizon) they fall in, cells in lexicographic order, ties by
    // caller id, for point sets given in no particular order.
    Grid g;
    perm.resize(n);
    inv.resize(n);
    if (reorder == 0 || !build_grid(g, n, x, delta)) {
        std::iota(perm.begin(), perm.end(), 0);
    } else {
        std::copy(g.items.begin(), g.items.end(), perm.begin());
    }
    for (int64_t p = 0; p < n; ++p) inv[perm[p]] = (int32_t)p;
}

void build_layout(int64_t n, const std::vector<int64_t>& off, const std::vector<int32_t>& idx,
                  const std::vector<int32_t>& perm, const std::vector<int32_t>& inv, int Q,
                  std::vector<int32_t>& nbr, std::vector<uint32_t>& bits,
                  std::vector<int32_t>& sw, std::vector<int32_t>& cnt)
{
    // Sliced ELL, slice height 32 (one warp): member m of node p = 32g + l at
    // nbr[(g*W + m)*32 + l]; bond flag word q at bits[(g*Q + q)*32 + l].
    const int64_t W = 32LL * Q;
    const int64_t ns = (n + 31) / 32;
    nbr.resize((size_t)(ns * W * 32));
    bits.assign((size_t)(ns * Q * 32), 0u);
    sw.assign((size_t)ns, 0);
    cnt.assign((size_t)(ns * 32), 0);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < ns; ++g) {
        std::vector<int32_t> row;
        int32_t width = 0;
        for (int l = 0; l < 32; ++l) {
            const int64_t p = g * 32 + l;
            row.clear();
            if (p < n) {
                const int64_t i = perm[p];
                for (int64_t k = off[i]; k < off[i + 1]; ++k) row.push_back(inv[idx[k]]);
                std::sort(row.begin(), row.end());
            }
            const int64_t m = (int64_t)row.size();
            for (int64_t k = 0; k < W; ++k)
                nbr[(g * W + k) * 32 + l] = k < m ? row[k] : (int32_t)p;
            for (int64_t k = 0; k < m; ++k)
                bits[(g * Q + (k >> 5)) * 32 + l] |= 1u << (k & 31);
            cnt[p] = (int32_t)m;
            width = std::max<int32_t>(width, (int32_t)m);
        }
        sw[g] = width;
    }
}

bool detect_lattice(int64_t n, const double* x, const std::vector<int64_t>& off,
                    const std::vector<int32_t>& idx, Lattice& L, std::vector<int32_t>& perm,
                    std::vector<int32_t>& inv)
{
    if (n < 2 || idx.empty()) return false;
    // spacing: the shortest bond
    double d2min = HUGE_VAL;
#pragma omp parallel for reduction(min : d2min) schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = off[i]; k < off[i + 1]; ++k) {
            const double* a = x + 3 * i;
            const double* b = x + 3 * (int64_t)idx[k];
            const double d2 = (b[0] - a[0]) * (b[0] - a[0]) + (b[1] - a[1]) * (b[1] - a[1]) +
                              (b[2] - a[2]) * (b[2] - a[2]);
            d2min = std::min(d2min, d2);
        }
    if (!(d2min > 0.0) || !std::isfinite(d2min)) return false;
    const double dx = std::sqrt(d2min);
    double lo[3];
    for (int a = 0; a < 3; ++a) lo[a] = x[a];
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) lo[a] = std::min(lo[a], x[3 * i + a]);
    // integer lattice coordinates, exact to 1e-9 dx
    std::vector<int64_t> ic(3 * n);
    int64_t N[3] = {0, 0, 0};
    const double tol = 1e-9 * dx;
    int bad = 0;
#pragma omp parallel for reduction(max : bad) schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            const double t = (x[3 * i + a] - lo[a]) / dx;
            const double r = std::nearbyint(t);
            const bool off_site = !(std::fabs(x[3 * i + a] - (lo[a] + r * dx)) <= tol) || r > 2.0e9;
            if (off_site) bad = 1;
            ic[3 * i + a] = off_site ? 0 : (int64_t)r;
        }
    if (bad) return false;
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) N[a] = std::max(N[a], ic[3 * i + a] + 1);
    if (N[0] * N[1] * N[2] != n) return false;
    perm.assign(n, -1);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t p = (ic[3 * i] * N[1] + ic[3 * i + 1]) * N[2] + ic[3 * i + 2];
        if (perm[p] != -1) return false;  // two nodes on one lattice site
        perm[p] = (int32_t)i;
    }
    // every bond a stencil offset, the largest |o|^2 = 9
    int qmax = 0;
#pragma omp parallel for reduction(max : qmax) schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = off[i]; k < off[i + 1]; ++k) {
            const int64_t j = idx[k];
            int q = 0;
            for (int a = 0; a < 3; ++a) {
                const int64_t d = ic[3 * j + a] - ic[3 * i + a];
                q += (d < -3 || d > 3) ? 100 : (int)(d * d);
            }
            qmax = std::max(qmax, q);
        }
    if (qmax != kStencilR2) return false;
    inv.assign(n, 0);
    for (int64_t p = 0; p < n; ++p) inv[perm[p]] = (int32_t)p;
    for (int a = 0; a < 3; ++a) L.N[a] = N[a];
    L.dx = dx;
    return true;
}

namespace {
// slot of each offset (o + 3 in [0, 7)^3), -1 outside the stencil
struct StencilLut {
    int s[343];
    StencilLut()
    {
        for (int& v : s) v = -1;
        for (int m = 0; m < kStencilSlots; ++m) {
            const Off3 o = stencil_offset(m);
            if (o.q == 0) continue;  // unused slot
            s[((o.x + 3) * 7 + (o.y + 3)) * 7 + (o.z + 3)] = m;
        }
    }
};
const StencilLut& stencil_lut()
{
    static const StencilLut lut;
    return lut;
}
}  // namespace

int stencil_slot(const Lattice& L, int64_t p, int64_t q)
{
    p -= L.first;
    q -= L.first;
    const int64_t pz = p % L.N[2], py = (p / L.N[2]) % L.N[1], px = p / (L.N[2] * L.N[1]);
    const int64_t qz = q % L.N[2], qy = (q / L.N[2]) % L.N[1], qx = q / (L.N[2] * L.N[1]);
    const int64_t ox = qx - px, oy = qy - py, oz = qz - pz;
    if (ox < -3 || ox > 3 || oy < -3 || oy > 3 || oz < -3 || oz > 3) return -1;
    return stencil_lut().s[((ox + 3) * 7 + (oy + 3)) * 7 + (oz + 3)];
}

void build_layout_stencil(int64_t n, const std::vector<int64_t>& off,
                          const std::vector<int32_t>& idx, const std::vector<int32_t>& perm,
                          const std::vector<int32_t>& inv, const std::vector<Lattice>& lats,
                          const std::vector<int32_t>* lat_of, std::vector<int32_t>& nbr,
                          std::vector<uint32_t>& bits, std::vector<int32_t>& sw,
                          std::vector<int32_t>& cnt)
{
    const int Q = kStencilSlots / 32;
    const int64_t W = 32LL * Q;
    const int64_t ns = (n + 31) / 32;
    nbr.resize((size_t)(ns * W * 32));
    bits.assign((size_t)(ns * Q * 32), 0u);
    sw.assign((size_t)ns, 0);
    cnt.assign((size_t)(ns * 32), 0);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < ns; ++g) {
        int32_t width = 0;
        for (int l = 0; l < 32; ++l) {
            const int64_t p = g * 32 + l;
            for (int64_t k = 0; k < W; ++k) nbr[(g * W + k) * 32 + l] = (int32_t)p;
            if (p >= n) continue;
            const int64_t i = perm[p];
            const Lattice& L = lats[lat_of ? (*lat_of)[p] : 0];
            for (int64_t k = off[i]; k < off[i + 1]; ++k) {
                const int32_t q = inv[idx[k]];
                const int m = stencil_slot(L, p, q);  // detect_lattice checked m >= 0
                nbr[(g * W + m) * 32 + l] = q;
                bits[(g * Q + (m >> 5)) * 32 + l] |= 1u << (m & 31);
                width = std::max(width, m + 1);
            }
            cnt[p] = (int32_t)(off[i + 1] - off[i]);
        }
        sw[g] = width;
    }
}

void slot_to_canonical(int64_t n, const std::vector<int64_t>& off, const std::vector<int32_t>& idx,
                       const std::vector<int32_t>& perm, const std::vector<int32_t>& nbr,
                       const std::vector<int32_t>& cnt, int Q, std::vector<int64_t>& pos)
{
    // pos[slot] = canonical CSR position of the bond in that SELL slot (-1 if unused)
    const int64_t W = 32LL * Q;
    const int64_t ns = (n + 31) / 32;
    pos.assign((size_t)(ns * W * 32), -1);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < n; ++p) {
        const int64_t g = p / 32, l = p % 32;
        const int64_t i = perm[p];
        const int32_t* b = idx.data() + off[i];
        const int32_t* e = idx.data() + off[i + 1];
        if (cnt[p] == 0) continue;
        for (int64_t m = 0; m < W; ++m) {
            const int64_t slot = (g * W + m) * 32 + l;
            if (nbr[slot] == (int32_t)p) continue;  // unused
            const int32_t j = perm[nbr[slot]];
            pos[slot] = off[i] + (std::lower_bound(b, e, j) - b);
        }
    }
}

std::string bc_classes(int64_t n, const uint8_t* type, const double* disp, const double* force,
                       const uint8_t* no_fail, std::vector<BcClass>& table,
                       std::vector<uint8_t>& cls, bool& has_nofail)
{
    struct Key {
        uint32_t mask;
        double v[6];
        bool operator<(const Key& o) const
        {
            if (mask != o.mask) return mask < o.mask;
            return std::memcmp(v, o.v, sizeof(v)) < 0;
        }
    };
    std::map<Key, int> ids;
    table.clear();
    cls.assign(n, 0);
    has_nofail = false;
    Key zero{};
    ids[zero] = 0;
    table.push_back(BcClass{});
    for (int64_t i = 0; i < n; ++i) {
        Key k{};
        for (int a = 0; a < 3; ++a) {
            if (type && type[3 * i + a] > 1) return "bc type must be 0 or 1";
            if (type && type[3 * i + a]) k.mask |= 1u << a;
            const double d = disp ? disp[3 * i + a] : 0.0;
            const double f = force ? force[3 * i + a] : 0.0;
            if (!std::isfinite(d) || !std::isfinite(f)) return "non-finite boundary value";
            k.v[a] = (k.mask & (1u << a)) ? d : 0.0;
            k.v[3 + a] = f;
        }
        if (no_fail && no_fail[i]) {
            k.mask |= 8u;
            has_nofail = true;
        }
        // normalise -0.0 so that equal tuples share a class
        for (double& v : k.v)
            if (v == 0.0) v = 0.0;
        auto it = ids.find(k);
        if (it == ids.end()) {
            if ((int)table.size() >= 256) return "more than 256 distinct boundary-condition tuples";
            BcClass b{};
            b.mask = k.mask;
            for (int a = 0; a < 3; ++a) {
                b.disp[a] = k.v[a];
                b.force[a] = k.v[3 + a];
            }
            it = ids.emplace(k, (int)table.size()).first;
            table.push_back(b);
        }
        cls[i] = (uint8_t)it->second;
    }
    return "";
}

void stiffness_factors(int64_t n, const double* x, const double* vol, double delta,
                       const int64_t* off, const int32_t* idx, int flags, double v0, double dx,
                       double* factor)
{
    // family volumes first (the correction needs both ends'), then one pass
    // over the bonds; each bond's factor depends only on its own two nodes
    std::vector<double> fam;
    if (flags & 2) {
        fam.resize((size_t)n);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            double v = 0.0;
            for (int64_t k = off[i]; k < off[i + 1]; ++k) v += vol[idx[k]];
            fam[(size_t)i] = v;
        }
    }
    const double inv_delta = 1.0 / delta;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = off[i]; k < off[i + 1]; ++k) {
            const int64_t j = idx[k];
            double f = 1.0;
            const double d0 = x[3 * j] - x[3 * i], d1 = x[3 * j + 1] - x[3 * i + 1],
                         d2 = x[3 * j + 2] - x[3 * i + 2];
            const double len = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
            if (flags & 1) f = 5.0 * (1.0 - len * inv_delta);
            if (flags & 2) f *= (2.0 * v0) / (fam[(size_t)i] + fam[(size_t)j]);
            if (flags & 4) f *= std::min(1.0, std::max(0.0, (delta + 0.5 * dx - len) / dx));
            factor[k] = f;
        }
    }
}

double stable_dt(int64_t n, const double* x, const double* vol, const std::vector<int64_t>& off,
                 const std::vector<int32_t>& idx, double c, double rho)
{
    // Silling & Askari (2005): dt < sqrt(2 rho / sum_j V_j c / |xi_ij|), minimum over nodes.
    double worst = 0.0;
#pragma omp parallel for reduction(max : worst) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = off[i]; k < off[i + 1]; ++k) {
            const int64_t j = idx[k];
            const double dx = x[3 * j] - x[3 * i], dy = x[3 * j + 1] - x[3 * i + 1],
                         dz = x[3 * j + 2] - x[3 * i + 2];
            s += vol[j] * c / std::sqrt(dx * dx + dy * dy + dz * dz);
        }
        worst = std::max(worst, s);
    }
    return worst > 0.0 ? std::sqrt(2.0 * rho / worst) : INFINITY;
}

}  // namespace pd
