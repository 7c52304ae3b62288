// Host-side model preparation (library internal).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "pd_internal.h"

namespace pd {

// Family of Eq. 9 by a uniform cell grid (edge = delta), rows ascending.
// Returns "" on success, else an error message.
std::string search_family(int64_t n, const double* x, double delta, std::vector<int64_t>& off,
                          std::vector<int32_t>& idx);
// Validate a caller-supplied canonical CSR family.
std::string check_family(int64_t n, const int64_t* off, const int32_t* idx);
// Remove bonds whose segment crosses a cut rectangle (initial notch, Section 6).
void apply_cuts(int64_t n, const double* x, const double* cuts, int32_t ncuts,
                std::vector<int64_t>& off, std::vector<int32_t>& idx);
// perm[p] = caller id of node position p; inv = inverse (reorder: 0 keep, 1 cells).
void spatial_order(int64_t n, const double* x, double delta, int reorder,
                   std::vector<int32_t>& perm, std::vector<int32_t>& inv);
// Sliced ELL (slice height 32, W = 32 Q slots), intact-bond bits, per-slice
// widths and per-node counts (padded to a multiple of 32 nodes).
void build_layout(int64_t n, const std::vector<int64_t>& off, const std::vector<int32_t>& idx,
                  const std::vector<int32_t>& perm, const std::vector<int32_t>& inv, int Q,
                  std::vector<int32_t>& nbr, std::vector<uint32_t>& bits,
                  std::vector<int32_t>& sw, std::vector<int32_t>& cnt);
// Regular cubic lattice: every node at lo + dx (ix, iy, iz), the n nodes filling
// an Nx x Ny x Nz box, and every bond of the family one of the stencil offsets
// (0 < |o|^2 <= 9, some bond with |o|^2 = 9).  On success perm / inv put the
// nodes in lattice order p = (ix Ny + iy) Nz + iz and true is returned.
struct Lattice {
    int64_t N[3] = {0, 0, 0};
    double dx = 0.0;
    int64_t first = 0;  // position of its first node in the library order (batches)
};
bool detect_lattice(int64_t n, const double* x, const std::vector<int64_t>& off,
                    const std::vector<int32_t>& idx, Lattice& L, std::vector<int32_t>& perm,
                    std::vector<int32_t>& inv);
// Stencil-ordered layout of lattice models (W = 128 slots, slot m holds
// stencil_offset(m)): absent members and unused slots hold the node itself
// with flag 0.  lats: one lattice per instance, in library order (a single
// model: one); lat_of[p]: the lattice of library position p (nullptr: lats[0]).
void build_layout_stencil(int64_t n, const std::vector<int64_t>& off,
                          const std::vector<int32_t>& idx, const std::vector<int32_t>& perm,
                          const std::vector<int32_t>& inv, const std::vector<Lattice>& lats,
                          const std::vector<int32_t>* lat_of, std::vector<int32_t>& nbr,
                          std::vector<uint32_t>& bits, std::vector<int32_t>& sw,
                          std::vector<int32_t>& cnt);
// Stencil slot of the bond from lattice node p to q (library positions, both in
// lattice L), -1 if the offset is not a stencil offset.
int stencil_slot(const Lattice& L, int64_t p, int64_t q);
// Canonical CSR position of every device slot (-1 for unused slots).  A slot
// is used when its neighbour differs from the node itself.
void slot_to_canonical(int64_t n, const std::vector<int64_t>& off, const std::vector<int32_t>& idx,
                       const std::vector<int32_t>& perm, const std::vector<int32_t>& nbr,
                       const std::vector<int32_t>& cnt, int Q, std::vector<int64_t>& pos);
// Deduplicate per-node (type, disp, force, no_fail) tuples into <= 256 classes.
std::string bc_classes(int64_t n, const uint8_t* type, const double* disp, const double* force,
                       const uint8_t* no_fail, std::vector<BcClass>& table,
                       std::vector<uint8_t>& cls, bool& has_nofail);
// Largest stable explicit time step (Silling & Askari 2005).
// Per directed bond (canonical order) factors multiplying the constant c:
// flags bit 0 conical micromodulus, factor 5 (1 - |xi|/delta); bit 1 volume
// surface correction 2 v0 / (V_i + V_j) with V_i the family volume of node i.
// bit 2: partial volume, the linear rule (delta + dx/2 - |xi|) / dx in [0, 1]
void stiffness_factors(int64_t n, const double* x, const double* vol, double delta,
                       const int64_t* off, const int32_t* idx, int flags, double v0, double dx,
                       double* factor);
double stable_dt(int64_t n, const double* x, const double* vol, const std::vector<int64_t>& off,
                 const std::vector<int32_t>& idx, double c, double rho);

}  // namespace pd
