// Host-side precompute and merge index maps (no CUDA here).
//
// Leaf operators (Section 3.1, Appendices A.1, B.1, C.1) for a reference leaf
// [-1, 1]^d; derivative-bearing operators are rescaled by 2/h per leaf size
// on the device.  Merge maps encode the block formulas of Appendices A.2, B.2
// and C.2 as per-child scatter tables (see MergeMaps).
#pragma once

#include <complex>
#include <cstdint>
#include <vector>

namespace hps {

struct Spectral1D {
  int p = 0, q = 0;
  std::vector<double> xc;     // p Chebyshev--Lobatto points, ascending, on [-1, 1]
  std::vector<double> xg;     // q Gauss--Legendre points, ascending
  std::vector<double> D;      // p x p differentiation matrix, row-major D[i*p + j]
  std::vector<double> DD;     // D * D, row-major
  std::vector<double> G2C;    // p x q interpolation Gauss -> Chebyshev, row-major
  std::vector<double> C2G;    // q x p interpolation Chebyshev -> Gauss, row-major
};

Spectral1D make_spectral(int p, int q);

// Reference DtN leaf operators (Algorithm "2D DtN local solve" and its 3D
// version).  Matrices are column-major for direct upload.
struct DtnLeafRef {
  int dim = 0, p = 0, q = 0;
  int npts = 0, ni = 0, ne = 0, nb = 0;
  std::vector<int> Ii;        // interior node indices (ascending)
  std::vector<int> Ie;        // boundary node indices (ascending)
  std::vector<int> prow;      // node -> row of P (index into Ie) or -1
  std::vector<double> P;      // ne x nb (column-major)
  std::vector<double> Qi;     // nb x ni : Q restricted to interior nodes, scale 1 (column-major)
  std::vector<double> QP;     // nb x nb : Q(:, Ie) * P, scale 1 (column-major)
};

DtnLeafRef make_dtn_leaf(const Spectral1D& s, int dim);

// Reference ItI leaf pieces (Algorithm "2D ItI local solve").
struct ItiLeafRef {
  int p = 0, q = 0, npts = 0, nown = 0, nb = 0;
  std::vector<int> own_node;  // 4(p-1) owned boundary nodes (rows of G and P)
  std::vector<int> own_axis;  // normal axis of the owning side
  std::vector<double> own_sgn;
  std::vector<int> Ii;        // interior nodes
  std::vector<double> P;      // nown x nb (column-major)
};

ItiLeafRef make_iti_leaf(const Spectral1D& s);

// QH = Q H for a leaf of side h with impedance eta: nb x p^2 complex
// (column-major).
std::vector<std::complex<double>> make_iti_QH(const Spectral1D& s, double hlen, double eta);

// Merge maps of one uniform level.  Children are in Morton order k.
// For child k and child boundary point i (canonical child order):
//   ext[k][i] >= 0 : index in the parent's canonical boundary (exterior point)
//   var[k][i] >= 0 : interior unknown that carries this point's incoming data
//                    (DtN: the shared Dirichlet value; ItI: the incoming
//                    impedance of child k)
//   eq[k][i]  >= 0 : ItI only: the interior unknown whose equation contains
//                    child k's outgoing impedance at this point (the
//                    neighbour's incoming unknown); DtN: equal to var.
// The ItI unknowns are ordered [incoming to even children | incoming to odd
// children] (parity of cx + cy), so that D = [[I, D12], [D21, I]].
// For the B X product: per child the lists of its exterior and interior
// points (child indices) and where they go.
struct MergeMaps {
  int dim = 0, nch = 0, n = 0;   // n = points per child side (2D) / face (3D)
  int nbc = 0, n_ext = 0, n_int = 0;
  bool iti = false;
  std::vector<int> ext, var, eq;           // [nch][nbc]
  std::vector<int> b_arow, b_crow;         // [nch][nbc/2]  child exterior points -> parent rows
  std::vector<int> b_acol, b_brow;         // [nch][nbc/2]  child interior points -> X rows (var)
  // ItI: per child its interior points' equation rows (eq), same order as
  // b_acol; the D12 / D21 products run over children {1, 2} (odd parity,
  // whose equations fill D12) and {0, 3} (even parity, D21).
  std::vector<int> i_eq;                   // [nch][nbc/2]
};

MergeMaps make_merge_maps(int dim, int n, bool iti);

// Leaf / root geometry (for hps_nodes).
void leaf_node_coords(int dim, const double* lo, const double* hi, int L, const Spectral1D& s,
                      double* out);
void root_boundary_coords(int dim, const double* lo, const double* hi, int L, const Spectral1D& s,
                          double* out);

}  // namespace hps
