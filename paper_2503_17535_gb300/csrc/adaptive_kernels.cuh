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

// A_b *= s[b] for nblocks consecutive blocks of `per` elements.
template <typename T>
cudaError_t scale_blocks(T* A, int64_t per, const double* s, int64_t nblocks, cudaStream_t st, Prof* pf);

// Refinement check: for each of nleaf leaves, err[leaf] = max over the 8 p^3
// child nodes of |f1 - L8f1 f0| (f0: p^3 values, f1: 8 p^3 values, x fastest,
// children in Morton order); I1 is the 2p x p child interpolation (row-major).
cudaError_t refine_check(const double* f0, const double* f1, int64_t nleaf, int p, const double* I1,
                         double* err, cudaStream_t st);

}  // namespace hps
