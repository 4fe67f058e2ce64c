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

// Task owning element e: the last task with elem0 <= e (binary search).
template <typename Task>
__device__ __forceinline__ int find_task(const Task* tasks, int ntask, int64_t e) {
  int lo = 0, hi = ntask - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].elem0 <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__device__ __forceinline__ T proj_col_value(const ProjTask<T>& tk, const double* C2F, int i, int jp) {
  const ProjDev& pj = tk.pj;
  if (jp == pj.np) return tk.src[i + (int64_t)pj.n * tk.ld_src];
  if (pj.kind[jp] == 0) return tk.src[i + (int64_t)pj.src[jp].x * tk.ld_src];
  const int fq = 4 * pj.q2;
  const int4 s = pj.src[jp];
  const int u = pj.u[jp];
  const int srcs[4] = {s.x, s.y, s.z, s.w};
  T v = T(0.0);
  for (int qd = 0; qd < 4; ++qd)
    for (int t = 0; t < pj.q2; ++t)
      v = fmac(v, tk.src[i + (int64_t)(srcs[qd] + t) * tk.ld_src], T(C2F[(qd * pj.q2 + t) + (int64_t)u * fq]));
  return v;
}

template <typename T>
__global__ void k_proj_cols_group(const ProjTask<T>* tasks, int ntask, int64_t total, const double* C2F) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const ProjTask<T>& tk = tasks[find_task(tasks, ntask, e)];
    const int64_t le = e - tk.elem0;
    const int i = (int)(le % tk.nrc), jp = (int)(le / tk.nrc);
    tk.out[i + (int64_t)jp * tk.ld_out] = proj_col_value(tk, C2F, i, jp);
  }
}

template <typename T>
__global__ void k_proj_rows_group(const ProjTask<T>* tasks, int ntask, int64_t total, const double* F2C) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const ProjTask<T>& tk = tasks[find_task(tasks, ntask, e)];
    const ProjDev& pj = tk.pj;
    const int64_t le = e - tk.elem0;
    const int ip = (int)(le % pj.np), j = (int)(le / pj.np);
    T v;
    if (pj.kind[ip] == 0) {
      v = tk.src[pj.src[ip].x + (int64_t)j * tk.ld_src];
    } else {
      const int4 s = pj.src[ip];
      const int u = pj.u[ip];
      const int srcs[4] = {s.x, s.y, s.z, s.w};
      v = T(0.0);
      for (int qd = 0; qd < 4; ++qd)
        for (int t = 0; t < pj.q2; ++t)
          v = fmac(v, tk.src[(srcs[qd] + t) + (int64_t)j * tk.ld_src], T(F2C[u + (int64_t)(qd * pj.q2 + t) * pj.q2]));
    }
    tk.out[ip + (int64_t)j * tk.ld_out] = v;
  }
}

template <typename T>
__global__ void k_zero_group(const ZeroTask<T>* tasks, int ntask, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const ZeroTask<T>& tk = tasks[find_task(tasks, ntask, e)];
    tk.p[e - tk.elem0] = T(0.0);
  }
}

__device__ inline void gather_add(double* p, double v) { atomicAdd(p, v); }

template <typename T>
__global__ void k_merge_gather_group(const GatherTask<T>* tasks, int ntask, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const GatherTask<T>& tk = tasks[find_task(tasks, ntask, e)];
    const int nbc = tk.nbc, ne = tk.n_ext, ni = tk.n_int;
    const int rc = (int)(e - tk.elem0);
    const int i = rc % nbc, j = rc / nbc;
    const T v = tk.Tc[rc];
    const int ei = tk.ext[i];
    const int ri = tk.var[i];
    if (j == nbc) {  // h column
      if (ei >= 0) tk.TP[ei + (int64_t)ne * ne] = v;
      else gather_add(&tk.R[ri + (int64_t)ni * ne], v);
      continue;
    }
    const int ej = tk.ext[j];
    const int vj = tk.var[j];
    if (ei >= 0) {
      if (ej >= 0) tk.TP[ei + (int64_t)ej * ne] = v;    // A (B is read in place)
    } else {
      if (ej >= 0) tk.R[ri + (int64_t)ej * ni] = v;     // C
      else gather_add(&tk.D[ri + (int64_t)vj * ni], v); // D: two addends per interface entry
    }
  }
}

template <typename T>
cudaError_t proj_cols_group(const ProjTask<T>* tasks, int ntask, int64_t total, const double* C2F, cudaStream_t st,
                            Prof* pf) {
  if (ntask <= 0 || total <= 0) return cudaSuccess;
  if (pf) pf->begin(st);
  k_proj_cols_group<T><<<grid_for(total), 256, 0, st>>>(tasks, ntask, total, C2F);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t proj_rows_group(const ProjTask<T>* tasks, int ntask, int64_t total, const double* F2C, cudaStream_t st,
                            Prof* pf) {
  if (ntask <= 0 || total <= 0) return cudaSuccess;
  if (pf) pf->begin(st);
  k_proj_rows_group<T><<<grid_for(total), 256, 0, st>>>(tasks, ntask, total, F2C);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t zero_group(const ZeroTask<T>* tasks, int ntask, int64_t total, cudaStream_t st, Prof* pf) {
  if (ntask <= 0 || total <= 0) return cudaSuccess;
  if (pf) pf->begin(st);
  k_zero_group<T><<<grid_for(total), 256, 0, st>>>(tasks, ntask, total);
  if (pf) pf->end(K_OTHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t merge_gather_group(const GatherTask<T>* tasks, int ntask, int64_t total, cudaStream_t st, Prof* pf) {
  if (ntask <= 0 || total <= 0) return cudaSuccess;
  if (pf) pf->begin(st);
  k_merge_gather_group<T><<<grid_for(total), 256, 0, st>>>(tasks, ntask, total);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) k_gint_group(const GintTask<T>* tasks, int ntask, int use_xp) {
  __shared__ T part[8][33];
  const int lane = threadIdx.x, cg = threadIdx.y;
  const int64_t tile = blockIdx.x;
  // task owning this tile (tile0 ascending)
  int lo = 0, hi = ntask - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].tile0 <= tile) lo = mid;
    else hi = mid - 1;
  }
  const GintTask<T>& tk = tasks[lo];
  const int rtiles = (tk.n_int + 31) / 32;
  const int64_t loc = tile - tk.tile0;
  const int r = (int)(loc % rtiles) * 32 + lane;
  const int c = (int)(loc / rtiles);
  const T* g = tk.gpar + (int64_t)c * tk.n_ext;
  T acc = T(0.0);
  if (r < tk.n_int)
    for (int j = cg; j < tk.n_ext; j += 8) acc = fmac(acc, tk.X[r + (int64_t)j * tk.n_int], g[j]);
  part[cg][lane] = acc;
  __syncthreads();
  if (cg == 0 && r < tk.n_int) {
    T s = use_xp ? tk.xp[r + (int64_t)c * tk.n_int] : tk.X[r + (int64_t)tk.n_ext * tk.n_int];
    for (int k = 0; k < 8; ++k) s = s + part[k][lane];
    tk.gint[r + (int64_t)c * tk.n_int] = -s;
  }
}

template <typename T>
__global__ void k_down_children_group(const ChildTask<T>* tasks, int ntask, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const ChildTask<T>& tk = tasks[find_task(tasks, ntask, e)];
    const int le = (int)(e - tk.elem0);
    const int i = le % tk.nbc, c = le / tk.nbc;
    const int ei = tk.ext[i];
    tk.out[le] = ei >= 0 ? tk.gpar[ei + (int64_t)c * tk.n_ext] : tk.gint[tk.var[i] + (int64_t)c * tk.n_int];
  }
}

template <typename T>
__global__ void k_gather_h_group(const ChildTask<T>* tasks, int ntask, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const ChildTask<T>& tk = tasks[find_task(tasks, ntask, e)];
    const int le = (int)(e - tk.elem0);
    const int i = le % tk.nbc, c = le / tk.nbc;
    const T v = tk.gint[le];
    const int ei = tk.ext[i];
    if (ei >= 0) tk.hp[ei + (int64_t)c * tk.n_ext] = v;
    else gather_add(&tk.r[tk.var[i] + (int64_t)c * tk.n_int], v);  // two children per interface entry
  }
}

template <typename T>
__global__ void k_unproject_group(const ProjTask<T>* tasks, int ntask, int64_t total, const double* C2F) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const ProjTask<T>& tk = tasks[find_task(tasks, ntask, e)];
    const ProjDev& pj = tk.pj;
    const int64_t le = e - tk.elem0;
    const int i = (int)(le % pj.n), c = (int)(le / pj.n);
    const int fq = 4 * pj.q2;
    T v;
    const int cp = pj.bcopy[i];
    if (cp >= 0) {
      v = tk.src[cp + (int64_t)c * tk.ld_src];
    } else {
      const int base = pj.bbase[i], row = pj.bquad[i] * pj.q2 + pj.bt[i];
      v = T(0.0);
      for (int u = 0; u < pj.q2; ++u)
        v = fmac(v, T(C2F[row + (int64_t)u * fq]), tk.src[base + u + (int64_t)c * tk.ld_src]);
    }
    tk.out[i + (int64_t)c * tk.ld_out] = v;
  }
}

template <typename T>
cudaError_t gint_group(const GintTask<T>* tasks, int ntask, int64_t tiles, int use_xp, cudaStream_t st, Prof* pf) {
  if (ntask <= 0 || tiles <= 0) return cudaSuccess;
  if (pf) pf->begin(st);
  k_gint_group<T><<<(unsigned)tiles, dim3(32, 8), 0, st>>>(tasks, ntask, use_xp);
  if (pf) pf->end(K_DOWN, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t down_children_group(const ChildTask<T>* tasks, int ntask, int64_t total, cudaStream_t st, Prof* pf) {
  if (ntask <= 0 || total <= 0) return cudaSuccess;
  if (pf) pf->begin(st);
  k_down_children_group<T><<<grid_for(total), 256, 0, st>>>(tasks, ntask, total);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t gather_h_group(const ChildTask<T>* tasks, int ntask, int64_t total, cudaStream_t st, Prof* pf) {
  if (ntask <= 0 || total <= 0) return cudaSuccess;
  if (pf) pf->begin(st);
  k_gather_h_group<T><<<grid_for(total), 256, 0, st>>>(tasks, ntask, total);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t unproject_group(const ProjTask<T>* tasks, int ntask, int64_t total, const double* C2F, cudaStream_t st,
                            Prof* pf) {
  if (ntask <= 0 || total <= 0) return cudaSuccess;
  if (pf) pf->begin(st);
  k_unproject_group<T><<<grid_for(total), 256, 0, st>>>(tasks, ntask, total, C2F);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template cudaError_t gint_group<double>(const GintTask<double>*, int, int64_t, int, cudaStream_t, Prof*);
template cudaError_t down_children_group<double>(const ChildTask<double>*, int, int64_t, cudaStream_t, Prof*);
template cudaError_t gather_h_group<double>(const ChildTask<double>*, int, int64_t, cudaStream_t, Prof*);
template cudaError_t unproject_group<double>(const ProjTask<double>*, int, int64_t, const double*, cudaStream_t,
                                             Prof*);
template cudaError_t proj_cols_group<double>(const ProjTask<double>*, int, int64_t, const double*, cudaStream_t,
                                             Prof*);
template cudaError_t proj_rows_group<double>(const ProjTask<double>*, int, int64_t, const double*, cudaStream_t,
                                             Prof*);
template cudaError_t zero_group<double>(const ZeroTask<double>*, int, int64_t, cudaStream_t, Prof*);
template cudaError_t merge_gather_group<double>(const GatherTask<double>*, int, int64_t, cudaStream_t, Prof*);

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
