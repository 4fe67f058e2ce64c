// Device kernels of the adaptive path (Section 4.2): 4-to-1 panel projection
// of a child's [T | h] onto the coarsened interfaces, interpolation of
// interface data back onto fine panels, per-block scaling, and the
// refinement check of Eq. "refinement check".
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "linalg.h"

namespace hps {

// Device copy of a ChildProj: per projected point kind (0 copy, 1 coarse
// point u of a fine group), u and the 4 source panel starts (int4); per child
// point the back map (copy source, or group base + quadrant + position).
struct ProjDev {
  int n = 0, np = 0, q2 = 0;
  const int* kind = nullptr;
  const int* u = nullptr;
  const int4* src = nullptr;
  const int* bcopy = nullptr;
  const int* bbase = nullptr;
  const int* bquad = nullptr;
  const int* bt = nullptr;
};

// out(:, j') = T Pc for j' < np, out(:, np) = T(:, n) (the h column):
// T is nrows x (n+1) with leading dimension ldT; out has leading dimension ldo.
template <typename T>
cudaError_t proj_cols(const T* Tc, int ldT, int nrows, const ProjDev& pj, const double* C2F, T* out,
                      int ldo, cudaStream_t st, Prof* pf);

// out(i', j) = (R A)(i', j) for the ncols columns of A (n rows, ld ldA).
template <typename T>
cudaError_t proj_rows(const T* A, int ldA, int ncols, const ProjDev& pj, const double* F2C, T* out,
                      int ldo, cudaStream_t st, Prof* pf);

// g(:, c) = Pc gp(:, c) for nrhs columns (gp: np x nrhs, g: n x nrhs).
template <typename T>
cudaError_t unproject(const T* gp, int ldgp, const ProjDev& pj, const double* C2F, T* g, int ldg,
                      int nrhs, cudaStream_t st, Prof* pf);

// Grouped forms for one tree level of an adaptive build: every (merge,
// child) pair of the level in one launch per step, tasks in a device array
// laid out element range after element range (elem0 ascending; a task's
// elements start at elem0).  Projections: a child's columns (src nrows x
// (n+1), out nrows x (np+1)) or rows (src n x ncols, out np x ncols).
template <typename T>
struct ProjTask {
  const T* src;
  int ld_src;
  int nrc;           // proj_cols: rows of src; proj_rows: columns
  ProjDev pj;
  T* out;
  int ld_out;
  int64_t elem0;
};
// Zero a buffer of n elements.
template <typename T>
struct ZeroTask {
  T* p;
  int64_t n;
  int64_t elem0;
};
// Scatter one child's projected [T | h] (nbc x (nbc+1)) into its merge's D,
// [C | h_int] and [A | h_ext] (DtN: two children add on every interface
// entry, so the atomic sums do not depend on their order).
template <typename T>
struct GatherTask {
  const T* Tc;
  int nbc, n_ext, n_int;
  const int* ext;
  const int* var;
  T* D;
  T* R;
  T* TP;
  int64_t elem0;
};
// Solve-pass tasks of one level (nrhs columns).  GintTask: gint = -(X_C gpar
// + x) of one merge (x: X's last column, or xp when not null); one CTA per
// 32-row tile.  ChildTask: one child's boundary data from its merge's gpar
// and gint (DtN), or a child's h gathered into its merge's r and hp.
template <typename T>
struct GintTask {
  const T* X;
  const T* xp;
  const T* gpar;
  T* gint;
  int n_ext, n_int, nrhs;
  int64_t tile0;
};
template <typename T>
struct ChildTask {
  const T* gpar;   // down: the merge's exterior data (n_ext x nrhs)
  const T* gint;   // down: its interior data (n_int x nrhs); up: the child's h (nbc x nrhs)
  T* out;          // down: the child's data (nbc x nrhs)
  T* r;            // up: the merge's r (n_int x nrhs, zeroed) and hp (n_ext x nrhs)
  T* hp;
  int nbc, n_ext, n_int, nrhs;
  const int* ext;
  const int* var;
  int64_t elem0;
};
template <typename T>
cudaError_t gint_group(const GintTask<T>* tasks, int ntask, int64_t tiles, int use_xp, cudaStream_t st, Prof* pf);
template <typename T>
cudaError_t down_children_group(const ChildTask<T>* tasks, int ntask, int64_t total, cudaStream_t st, Prof* pf);
template <typename T>
cudaError_t gather_h_group(const ChildTask<T>* tasks, int ntask, int64_t total, cudaStream_t st, Prof* pf);
// Unprojection of every child of a level: ProjTask with src = the projected
// data (np x nrhs), nrc = nrhs, out = the child's data (n x nrhs, ld_out).
template <typename T>
cudaError_t unproject_group(const ProjTask<T>* tasks, int ntask, int64_t total, const double* C2F, cudaStream_t st,
                            Prof* pf);

template <typename T>
cudaError_t proj_cols_group(const ProjTask<T>* tasks, int ntask, int64_t total, const double* C2F, cudaStream_t st,
                            Prof* pf);
template <typename T>
cudaError_t proj_rows_group(const ProjTask<T>* tasks, int ntask, int64_t total, const double* F2C, cudaStream_t st,
                            Prof* pf);
template <typename T>
cudaError_t zero_group(const ZeroTask<T>* tasks, int ntask, int64_t total, cudaStream_t st, Prof* pf);
template <typename T>
cudaError_t merge_gather_group(const GatherTask<T>* tasks, int ntask, int64_t total, cudaStream_t st, Prof* pf);

// A_b *= s[b] for nblocks consecutive blocks of `per` elements.
template <typename T>
cudaError_t scale_blocks(T* A, int64_t per, const double* s, int64_t nblocks, cudaStream_t st, Prof* pf);

// Refinement check: for each of nleaf leaves, err[leaf] = max over the 8 p^3
// child nodes of |f1 - L8f1 f0| (f0: p^3 values, f1: 8 p^3 values, x fastest,
// children in Morton order); I1 is the 2p x p child interpolation (row-major).
cudaError_t refine_check(const double* f0, const double* f1, int64_t nleaf, int p, const double* I1,
                         double* err, cudaStream_t st);

}  // namespace hps
