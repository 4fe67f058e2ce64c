// HPS-specific device kernels: leaf assembly (Section 3.2), merge gathers
// (Section 3.3, Appendices A.2 / B.2 / C.2), downward pass and leaf output
// (Section 3.4).  Declarations; definitions in hps_kernels.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "linalg.h"

namespace hps {

// Geometry / operator constants needed by the leaf kernels.
struct LeafConsts {
  int dim, p, npts, ni, ne, nb, nown;
  double s;         // 2 / leaf side
  const double* sleaf;  // per-leaf 2 / side (adaptive trees) or null
  double eta;       // ItI impedance parameter
  const double* D;  // p x p row-major reference differentiation matrix
  const double* DD; // D*D row-major
  const int* Ii;    // interior nodes (ni)
  const int* prow;  // node -> row of P (DtN) or -1
  const int* iidx;  // node -> interior index or -1
  const double* P;  // DtN: ne x nb; ItI: nown x nb (column-major)
  const int* own_node;
  const int* own_axis;
  const double* own_sgn;
};

struct Coeffs {
  const double* a;   // may be null (a = 1)
  const double* b[3];
  const double* c;   // may be null (c = 0)
};

// DtN leaf: Lii (nl x ni x ni) and RHS = [L_ie P | -f_i] (nl x ni x (nb+1)).
cudaError_t leaf_dtn_assemble(const LeafConsts& k, int64_t nl, Coeffs cf, const double* f,
                              double* Lii, double* rhs, cudaStream_t st, Prof* pf);
// ItI leaf: B = [G; L(I_i, :)] (nl x npts x npts) and RHS = [[P, 0], [0, f_i]].
cudaError_t leaf_iti_assemble(const LeafConsts& k, int64_t nl, Coeffs cf, const cplx* f,
                              cplx* B, cplx* rhs, cudaStream_t st, Prof* pf);
// Pieces of the ItI interior elimination: L(I_i, I_i) (as for DtN leaves),
// L(I_i, boundary nodes in owner order) (nl x ni x nown) and the right-hand
// sides [[P, 0], [0, f_i]] alone.
cudaError_t leaf_assemble_Lii(const LeafConsts& k, int64_t nl, Coeffs cf, double* Lii, cudaStream_t st, Prof* pf);
cudaError_t leaf_iti_Lie(const LeafConsts& k, int64_t nl, Coeffs cf, double* Lie, cudaStream_t st, Prof* pf);
cudaError_t leaf_iti_rhs(const LeafConsts& k, int64_t nl, const cplx* f, cplx* rhs, cudaStream_t st, Prof* pf);
// Bounds of the coefficients over n nodes: h_out = (min a, max |b_k|, max c)
// (defaults a = 1, b = 0, c = 0 for missing arrays); d_out holds 192
// doubles of device scratch.  Synchronises the stream.
cudaError_t coef_bounds(Coeffs cf, int dim, int64_t n, double* d_out, double* h_out, cudaStream_t st);
// Right-hand sides of the upward particular pass: DtN -f_i; ItI [0; f_i].
// f is [nrhs][nl][npts]; out is per leaf an (rows x nrhs) column-major block.
template <typename T>
cudaError_t leaf_particular_rhs(const LeafConsts& k, int64_t nl, int nrhs, const T* f, T* out,
                                bool iti, cudaStream_t st, Prof* pf);
// T|h init for DtN leaves: C = s * [QP | 0] (nb x (nb+1)) per leaf.
cudaError_t leaf_dtn_init_T(const double* QP, int nb, double s, int64_t nl, double* TH,
                            cudaStream_t st, Prof* pf);

// Merge gather of one level: children's [T | h] (nbc x (nbc+1), contiguous
// per child in Morton order, `cstride` elements apart) into D (n_int x n_int),
// R = [C | h_int] (n_int x (n_ext+1)) and TP = [A | h_ext] (n_ext x (n_ext+1)).
// DtN rows use `var` (two children add on interfaces); ItI rows use `eq`.
template <typename T>
cudaError_t merge_gather(const T* Tc, int64_t cstride, int nmerge, int nch, int nbc, int n_ext,
                         int n_int, const int* ext, const int* var, const int* eq, bool iti, T* D,
                         T* R, T* TP, cudaStream_t st, Prof* pf);

// Gather children's h (nrhs columns; child block = nbc x nrhs) into
// r (n_int x nrhs per merge, must be zeroed for DtN) and hp (n_ext x nrhs).
template <typename T>
cudaError_t merge_gather_h(const T* hc, int nmerge, int nch, int nbc, int n_ext, int n_int,
                           int nrhs, const int* ext, const int* var, const int* eq, bool iti, T* r,
                           T* hp, cudaStream_t st, Prof* pf);

// Downward step: gint = -(X_C g + xpart) for every merge (nrhs columns), then
// the children's boundary data.  X is n_int x (n_ext+1) per merge; xpart is
// either X's last column (xp == null) or a separate n_int x nrhs block.
template <typename T>
cudaError_t down_level(const T* X, const T* xp, const T* gpar, int nmerge, int nch, int nbc,
                       int n_ext, int n_int, int nrhs, const int* ext, const int* var, T* gint,
                       T* gchild, cudaStream_t st, Prof* pf);

// The two halves of down_level, for merges whose children differ in size.
template <typename T>
cudaError_t down_gint(const T* X, const T* xp, const T* gpar, int nmerge, int n_ext, int n_int, int nrhs,
                      T* gint, cudaStream_t st, Prof* pf);
template <typename T>
cudaError_t down_children(const T* gpar, const T* gint, int nmerge, int nch, int nbc, int n_ext, int n_int,
                          int nrhs, const int* ext, const int* var, T* gchild, cudaStream_t st, Prof* pf);

// Leaf output u = Y g + v for every leaf and right-hand side.
//   DtN: u(I_e) = P g, u(I_i) = -(X_Y g + xpart)   (X = ni x (nb+1))
//   ItI: u = X_Y g + xpart                          (X = npts x (nb+1))
// u is [nrhs][nl][npts]; g is per leaf an nb x nrhs block.
template <typename T>
cudaError_t leaf_output(const LeafConsts& k, int64_t nl, int nrhs, const T* X, const T* xp,
                        const T* g, T* u, bool iti, cudaStream_t st, Prof* pf);

// Grouped downward pass and leaf output: one launch serves the same level
// (counted from each tree's root) of up to kMaxGroup different operators,
// whose depths, orders and sizes may all differ (Section 3.4, Algorithm
// "down pass", applied to many trees at once).  Each task carries its own
// pointers and sizes; the launch's tiles / elements are laid out task after
// task and every CTA or thread finds its task from the prefix offsets.
constexpr int kMaxGroup = 24;

template <typename T>
struct DownTask {
  const T* X;        // n_int x (n_ext+1) per merge; the last column is x
  const T* gpar;     // n_ext x nrhs per merge
  T* gint;           // n_int x nrhs per merge
  T* gchild;         // children's boundary data, nbc x nrhs per child
  const int* ext;
  const int* var;
  int nmerge, nch, nbc, n_ext, n_int, nrhs;
  int64_t tile0;     // first 32-row tile of this task in the gint launch
  int64_t elem0;     // first element of this task in the children launch
};
template <typename T>
struct DownGroup {
  int n;
  int64_t tiles, elems;  // totals
  DownTask<T> t[kMaxGroup];
};
template <typename T>
struct LeafTask {
  LeafConsts k;
  int64_t nl;
  int nrhs;
  const T* X;
  const T* g;        // per leaf nb x nrhs
  T* u;              // [nrhs][nl][npts]
  int64_t elem0;
};
template <typename T>
struct LeafGroup {
  int n;
  bool iti;
  int64_t elems;
  LeafTask<T> t[kMaxGroup];
};
// gint of every task, then the children's data (two launches).
template <typename T>
cudaError_t down_level_group(const DownGroup<T>& grp, cudaStream_t st);
// u = Y g + v (build-time source) for every task (one launch).
template <typename T>
cudaError_t leaf_output_group(const LeafGroup<T>& grp, cudaStream_t st);

// Copy rows [r0, r0+m) of src blocks into dst blocks (same column count).
template <typename T>
cudaError_t copy_block(const T* src, int64_t sstride, int sld, T* dst, int64_t dstride, int dld,
                       int m, int ncols, int batch, cudaStream_t st, Prof* pf);

// Scatter g_root ([nrhs][n]) into the top-level layout (n x nrhs) or gather
// u; also used to negate.  Generic strided 2D copy with optional negation.
template <typename T>
cudaError_t scale_copy(const T* src, T* dst, int64_t n, double alpha, cudaStream_t st, Prof* pf);

}  // namespace hps
