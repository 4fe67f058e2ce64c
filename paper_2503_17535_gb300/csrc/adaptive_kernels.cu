// Adaptive-path kernels: panel projections, interpolation back to fine
// panels, block scaling and the refinement check.
#include "adaptive_kernels.cuh"

#include <algorithm>

namespace hps {

namespace {
inline int grid_for(int64_t total, int threads = 256) {
  int64_t b = (total + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 65535 * 8));
}
}  // namespace

template <typename T>
__global__ void k_proj_cols(const T* Tc, int ldT, int nrows, ProjDev pj, const double* C2F, T* out, int ldo) {
  const int64_t total = (int64_t)nrows * (pj.np + 1);
  const int fq = 4 * pj.q2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % nrows), jp = (int)(e / nrows);
    T v;
    if (jp == pj.np) {
      v = Tc[i + (int64_t)pj.n * ldT];
    } else if (pj.kind[jp] == 0) {
      v = Tc[i + (int64_t)pj.src[jp].x * ldT];
    } else {
      const int4 s = pj.src[jp];
      const int u = pj.u[jp];
      const int srcs[4] = {s.x, s.y, s.z, s.w};
      v = T(0.0);
      for (int qd = 0; qd < 4; ++qd)
        for (int t = 0; t < pj.q2; ++t)
          v = fmac(v, Tc[i + (int64_t)(srcs[qd] + t) * ldT], T(C2F[(qd * pj.q2 + t) + (int64_t)u * fq]));
    }
    out[i + (int64_t)jp * ldo] = v;
  }
}

template <typename T>
cudaError_t proj_cols(const T* Tc, int ldT, int nrows, const ProjDev& pj, const double* C2F, T* out, int ldo,
                      cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_proj_cols<T><<<grid_for((int64_t)nrows * (pj.np + 1)), 256, 0, st>>>(Tc, ldT, nrows, pj, C2F, out, ldo);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_proj_rows(const T* A, int ldA, int ncols, ProjDev pj, const double* F2C, T* out, int ldo) {
  const int64_t total = (int64_t)pj.np * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int ip = (int)(e % pj.np), j = (int)(e / pj.np);
    T v;
    if (pj.kind[ip] == 0) {
      v = A[pj.src[ip].x + (int64_t)j * ldA];
    } else {
      const int4 s = pj.src[ip];
      const int u = pj.u[ip];
      const int srcs[4] = {s.x, s.y, s.z, s.w};
      v = T(0.0);
      for (int qd = 0; qd < 4; ++qd)
        for (int t = 0; t < pj.q2; ++t)
          v = fmac(v, A[(srcs[qd] + t) + (int64_t)j * ldA], T(F2C[u + (int64_t)(qd * pj.q2 + t) * pj.q2]));
    }
    out[ip + (int64_t)j * ldo] = v;
  }
}

template <typename T>
cudaError_t proj_rows(const T* A, int ldA, int ncols, const ProjDev& pj, const double* F2C, T* out, int ldo,
                      cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_proj_rows<T><<<grid_for((int64_t)pj.np * ncols), 256, 0, st>>>(A, ldA, ncols, pj, F2C, out, ldo);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_unproject(const T* gp, int ldgp, ProjDev pj, const double* C2F, T* g, int ldg, int nrhs) {
  const int64_t total = (int64_t)pj.n * nrhs;
  const int fq = 4 * pj.q2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % pj.n), c = (int)(e / pj.n);
    T v;
    const int cp = pj.bcopy[i];
    if (cp >= 0) {
      v = gp[cp + (int64_t)c * ldgp];
    } else {
      const int base = pj.bbase[i], row = pj.bquad[i] * pj.q2 + pj.bt[i];
      v = T(0.0);
      for (int u = 0; u < pj.q2; ++u) v = fmac(v, T(C2F[row + (int64_t)u * fq]), gp[base + u + (int64_t)c * ldgp]);
    }
    g[i + (int64_t)c * ldg] = v;
  }
}

template <typename T>
cudaError_t unproject(const T* gp, int ldgp, const ProjDev& pj, const double* C2F, T* g, int ldg, int nrhs,
                      cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_unproject<T><<<grid_for((int64_t)pj.n * nrhs), 256, 0, st>>>(gp, ldgp, pj, C2F, g, ldg, nrhs);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_scale_blocks(T* A, int64_t per, const double* s, int64_t nblocks) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * nblocks;
       e += (int64_t)gridDim.x * blockDim.x)
    A[e] = scale(A[e], s[e / per]);
}

template <typename T>
cudaError_t scale_blocks(T* A, int64_t per, const double* s, int64_t nblocks, cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_scale_blocks<T><<<grid_for(per * nblocks), 256, 0, st>>>(A, per, s, nblocks);
  if (pf) pf->end(K_OTHER, 0.0, st);
  return cudaGetLastError();
}

// One block per leaf; each thread takes child nodes and evaluates the tensor
// interpolant of the leaf's p^3 values there (separable sums), then a block
// max-reduction.
__global__ void k_refine_check(const double* f0, const double* f1, int64_t nleaf, int p, const double* I1,
                               double* err) {
  extern __shared__ double sm[];
  double* F = sm;                 // p^3
  double* red = sm + p * p * p;   // blockDim.x
  const int npts = p * p * p;
  for (int64_t leaf = blockIdx.x; leaf < nleaf; leaf += gridDim.x) {
    __syncthreads();
    for (int e = threadIdx.x; e < npts; e += blockDim.x) F[e] = f0[leaf * npts + e];
    __syncthreads();
    double mx = 0.0;
    for (int e = threadIdx.x; e < 8 * npts; e += blockDim.x) {
      const int c = e / npts, node = e % npts;
      const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
      const int ax = cx * p + node % p, ay = cy * p + (node / p) % p, az = cz * p + node / (p * p);
      double v = 0.0;
      for (int k = 0; k < p; ++k) {
        double vy = 0.0;
        for (int j = 0; j < p; ++j) {
          double vx = 0.0;
          for (int i = 0; i < p; ++i) vx = fma(I1[ax * p + i], F[i + p * (j + p * k)], vx);
          vy = fma(I1[ay * p + j], vx, vy);
        }
        v = fma(I1[az * p + k], vy, v);
      }
      mx = fmax(mx, fabs(f1[leaf * 8 * npts + e] - v));
    }
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
      if (threadIdx.x < s2) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s2]);
      __syncthreads();
    }
    if (threadIdx.x == 0) err[leaf] = red[0];
  }
}

cudaError_t refine_check(const double* f0, const double* f1, int64_t nleaf, int p, const double* I1, double* err,
                         cudaStream_t st) {
  if (nleaf <= 0) return cudaSuccess;
  const int threads = 256;
  const size_t sm = ((size_t)p * p * p + threads) * sizeof(double);
  k_refine_check<<<(int)std::min<int64_t>(nleaf, 65535), threads, sm, st>>>(f0, f1, nleaf, p, I1, err);
  return cudaGetLastError();
}

#define HPS_AINST(T)                                                                                    \
  template cudaError_t proj_cols<T>(const T*, int, int, const ProjDev&, const double*, T*, int,          \
                                    cudaStream_t, Prof*);                                                \
  template cudaError_t proj_rows<T>(const T*, int, int, const ProjDev&, const double*, T*, int,          \
                                    cudaStream_t, Prof*);                                                \
  template cudaError_t unproject<T>(const T*, int, const ProjDev&, const double*, T*, int, int,          \
                                    cudaStream_t, Prof*);                                                \
  template cudaError_t scale_blocks<T>(T*, int64_t, const double*, int64_t, cudaStream_t, Prof*);

HPS_AINST(double)
HPS_AINST(cplx)

}  // namespace hps
