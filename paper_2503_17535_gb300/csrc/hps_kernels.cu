// HPS-specific device kernels (leaf assembly, merge gathers, downward pass,
// leaf output).  These are gather/scatter and small dot-product kernels; the
// dense FP64 work (LU, triangular solves, GEMM) lives in linalg.cu.
#include "hps_kernels.cuh"

#include <algorithm>

namespace hps {

namespace {

inline int grid_for(int64_t total, int threads = 256, int cap = 65535 * 8) {
  int64_t b = (total + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

__device__ inline void coords(int dim, int p, int idx, int* c) {
  c[0] = idx % p;
  c[1] = (idx / p) % p;
  c[2] = dim == 3 ? idx / (p * p) : 0;
}

// Entry (i, j) of the leaf operator a Lap + sum_k b_k d_k + c (Section 3.2)
// on the tensor Chebyshev grid: nonzero only when i and j differ along at
// most one axis.
__device__ inline double L_entry(const LeafConsts& k, double s, double a, const double* bk, double c,
                                 int i, int j) {
  int ci[3], cj[3];
  coords(k.dim, k.p, i, ci);
  coords(k.dim, k.p, j, cj);
  int ndiff = 0, dax = -1;
  for (int ax = 0; ax < k.dim; ++ax)
    if (ci[ax] != cj[ax]) { ++ndiff; dax = ax; }
  if (ndiff > 1) return 0.0;
  double v = 0.0;
  const double s2 = s * s;
  for (int ax = 0; ax < k.dim; ++ax) {
    if (ndiff == 1 && ax != dax) continue;
    const int e = ci[ax] * k.p + cj[ax];
    v = fma(a * s2, k.DD[e], v);
    v = fma(bk[ax] * s, k.D[e], v);
  }
  if (ndiff == 0) v += c;
  return v;
}

__device__ inline void load_coeffs(const Coeffs& cf, int64_t at, int dim, double* a, double* b,
                                   double* c) {
  *a = cf.a ? cf.a[at] : 1.0;
  for (int ax = 0; ax < 3; ++ax) b[ax] = (ax < dim && cf.b[ax]) ? cf.b[ax][at] : 0.0;
  *c = cf.c ? cf.c[at] : 0.0;
}

}  // namespace

// --------------------------------------------------------------- leaves ----

__global__ void k_leaf_dtn_Lii(LeafConsts k, int64_t nl, Coeffs cf, double* Lii) {
  const int64_t per = (int64_t)k.ni * k.ni;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * per;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t leaf = e / per;
    const int rc = (int)(e % per);
    const int r = rc % k.ni, c = rc / k.ni;
    const int i = k.Ii[r], j = k.Ii[c];
    double a, b[3], cc;
    load_coeffs(cf, leaf * k.npts + i, k.dim, &a, b, &cc);
    const double s = k.sleaf ? k.sleaf[leaf] : k.s;
    Lii[e] = L_entry(k, s, a, b, cc, i, j);
  }
}

__global__ void k_leaf_dtn_rhs(LeafConsts k, int64_t nl, Coeffs cf, const double* f, double* rhs) {
  const int ncol = k.nb + 1;
  const int64_t per = (int64_t)k.ni * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * per;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t leaf = e / per;
    const int rc = (int)(e % per);
    const int r = rc % k.ni, col = rc / k.ni;
    const int i = k.Ii[r];
    if (col == k.nb) {
      rhs[e] = f ? -f[leaf * k.npts + i] : 0.0;
      continue;
    }
    double a, b[3], cc;
    load_coeffs(cf, leaf * k.npts + i, k.dim, &a, b, &cc);
    const double s = k.sleaf ? k.sleaf[leaf] : k.s;
    int ci[3];
    coords(k.dim, k.p, i, ci);
    double acc = 0.0;
    for (int ax = 0; ax < k.dim; ++ax) {
      for (int end = 0; end < 2; ++end) {
        int cj[3] = {ci[0], ci[1], ci[2]};
        cj[ax] = end ? k.p - 1 : 0;
        const int j = cj[0] + k.p * (cj[1] + k.p * cj[2]);
        const int pr = k.prow[j];
        const int el = ci[ax] * k.p + cj[ax];
        const double lij = fma(a * s * s, k.DD[el], b[ax] * s * k.D[el]);
        acc = fma(lij, k.P[pr + (int64_t)col * k.ne], acc);
      }
    }
    rhs[e] = acc;
  }
}

cudaError_t leaf_dtn_assemble(const LeafConsts& k, int64_t nl, Coeffs cf, const double* f,
                              double* Lii, double* rhs, cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_leaf_dtn_Lii<<<grid_for(nl * k.ni * k.ni), 256, 0, st>>>(k, nl, cf, Lii);
  if (pf) pf->end(K_ASSEMBLE, 0.0, st);
  if (pf) pf->begin(st);
  k_leaf_dtn_rhs<<<grid_for(nl * k.ni * (k.nb + 1)), 256, 0, st>>>(k, nl, cf, f, rhs);
  if (pf) pf->end(K_ASSEMBLE, 2.0 * 2 * k.dim * (double)nl * k.ni * k.nb, st);
  return cudaGetLastError();
}

__global__ void k_leaf_iti_B(LeafConsts k, int64_t nl, Coeffs cf, cplx* B) {
  const int n = k.npts;
  const int64_t per = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * per;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t leaf = e / per;
    const int rc = (int)(e % per);
    const int r = rc % n, j = rc / n;
    cplx v(0.0, 0.0);
    if (r < k.nown) {
      // incoming impedance row: sgn * s * d/dx_axis + i eta at the owned node
      const int node = k.own_node[r], ax = k.own_axis[r];
      int ci[3], cj[3];
      coords(k.dim, k.p, node, ci);
      coords(k.dim, k.p, j, cj);
      bool same = true;
      for (int a2 = 0; a2 < k.dim; ++a2)
        if (a2 != ax && ci[a2] != cj[a2]) same = false;
      if (same) v.re = k.own_sgn[r] * k.s * k.D[ci[ax] * k.p + cj[ax]];
      if (j == node) v.im = k.eta;
    } else {
      const int i = k.Ii[r - k.nown];
      double a, b[3], cc;
      load_coeffs(cf, leaf * k.npts + i, k.dim, &a, b, &cc);
      v.re = L_entry(k, k.s, a, b, cc, i, j);
    }
    B[e] = v;
  }
}

__global__ void k_leaf_iti_rhs(LeafConsts k, int64_t nl, const cplx* f, cplx* rhs) {
  const int n = k.npts, ncol = k.nb + 1;
  const int64_t per = (int64_t)n * ncol;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * per;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t leaf = e / per;
    const int rc = (int)(e % per);
    const int r = rc % n, col = rc / n;
    cplx v(0.0, 0.0);
    if (col < k.nb) {
      if (r < k.nown) v = cplx(k.P[r + (int64_t)col * k.nown], 0.0);
    } else if (r >= k.nown && f) {
      v = f[leaf * k.npts + k.Ii[r - k.nown]];
    }
    rhs[e] = v;
  }
}

// L(I_i, boundary nodes in owner order): the interior rows of the leaf
// operator on the boundary columns, for the ItI interior elimination.
__global__ void k_leaf_iti_Lie(LeafConsts k, int64_t nl, Coeffs cf, double* Lie) {
  const int64_t per = (int64_t)k.ni * k.nown;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * per;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t leaf = e / per;
    const int rc = (int)(e % per);
    const int r = rc % k.ni, c = rc / k.ni;
    const int i = k.Ii[r], j = k.own_node[c];
    double a, b[3], cc;
    load_coeffs(cf, leaf * k.npts + i, k.dim, &a, b, &cc);
    Lie[e] = L_entry(k, k.s, a, b, cc, i, j);
  }
}

// Per-block bounds of the coefficients: out[3 * block + {0, 1, 2}] =
// (min a, max |b|, max c) over this block's share of the nodes.
__global__ void k_coef_bounds(Coeffs cf, int dim, int64_t n, double* out) {
  __shared__ double sa[256], sb[256], sc[256];
  double amin = 1e300, bmax = 0.0, cmax = -1e300;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    amin = fmin(amin, cf.a ? cf.a[e] : 1.0);
    for (int ax = 0; ax < dim; ++ax) bmax = fmax(bmax, cf.b[ax] ? fabs(cf.b[ax][e]) : 0.0);
    cmax = fmax(cmax, cf.c ? cf.c[e] : 0.0);
  }
  sa[threadIdx.x] = amin;
  sb[threadIdx.x] = bmax;
  sc[threadIdx.x] = cmax;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sa[threadIdx.x] = fmin(sa[threadIdx.x], sa[threadIdx.x + o]);
      sb[threadIdx.x] = fmax(sb[threadIdx.x], sb[threadIdx.x + o]);
      sc[threadIdx.x] = fmax(sc[threadIdx.x], sc[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[3 * blockIdx.x] = sa[0];
    out[3 * blockIdx.x + 1] = sb[0];
    out[3 * blockIdx.x + 2] = sc[0];
  }
}

cudaError_t leaf_assemble_Lii(const LeafConsts& k, int64_t nl, Coeffs cf, double* Lii, cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_leaf_dtn_Lii<<<grid_for(nl * k.ni * k.ni), 256, 0, st>>>(k, nl, cf, Lii);
  if (pf) pf->end(K_ASSEMBLE, 0.0, st);
  return cudaGetLastError();
}

cudaError_t leaf_iti_Lie(const LeafConsts& k, int64_t nl, Coeffs cf, double* Lie, cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_leaf_iti_Lie<<<grid_for(nl * k.ni * k.nown), 256, 0, st>>>(k, nl, cf, Lie);
  if (pf) pf->end(K_ASSEMBLE, 0.0, st);
  return cudaGetLastError();
}

cudaError_t leaf_iti_rhs(const LeafConsts& k, int64_t nl, const cplx* f, cplx* rhs, cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_leaf_iti_rhs<<<grid_for(nl * k.npts * (k.nb + 1)), 256, 0, st>>>(k, nl, f, rhs);
  if (pf) pf->end(K_ASSEMBLE, 0.0, st);
  return cudaGetLastError();
}

cudaError_t coef_bounds(Coeffs cf, int dim, int64_t n, double* d_out, double* h_out, cudaStream_t st) {
  constexpr int nblk = 64;
  k_coef_bounds<<<nblk, 256, 0, st>>>(cf, dim, n, d_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  double tmp[3 * nblk];
  if ((e = cudaMemcpyAsync(tmp, d_out, sizeof(tmp), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  h_out[0] = 1e300; h_out[1] = 0.0; h_out[2] = -1e300;
  for (int b = 0; b < nblk; ++b) {
    h_out[0] = std::min(h_out[0], tmp[3 * b]);
    h_out[1] = std::max(h_out[1], tmp[3 * b + 1]);
    h_out[2] = std::max(h_out[2], tmp[3 * b + 2]);
  }
  return cudaSuccess;
}

cudaError_t leaf_iti_assemble(const LeafConsts& k, int64_t nl, Coeffs cf, const cplx* f, cplx* B,
                              cplx* rhs, cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_leaf_iti_B<<<grid_for(nl * k.npts * k.npts), 256, 0, st>>>(k, nl, cf, B);
  if (pf) pf->end(K_ASSEMBLE, 0.0, st);
  if (pf) pf->begin(st);
  k_leaf_iti_rhs<<<grid_for(nl * k.npts * (k.nb + 1)), 256, 0, st>>>(k, nl, f, rhs);
  if (pf) pf->end(K_ASSEMBLE, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_leaf_particular_rhs(LeafConsts k, int64_t nl, int nrhs, const T* f, T* out, bool iti) {
  const int rows = iti ? k.npts : k.ni;
  const int64_t per = (int64_t)rows * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * per;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t leaf = e / per;
    const int rc = (int)(e % per);
    const int r = rc % rows, c = rc / rows;
    const int64_t fo = ((int64_t)c * nl + leaf) * k.npts;
    T v = T(0.0);
    if (!iti) v = -f[fo + k.Ii[r]];
    else if (r >= k.nown) v = f[fo + k.Ii[r - k.nown]];
    out[e] = v;
  }
}

template <typename T>
cudaError_t leaf_particular_rhs(const LeafConsts& k, int64_t nl, int nrhs, const T* f, T* out,
                                bool iti, cudaStream_t st, Prof* pf) {
  const int rows = iti ? k.npts : k.ni;
  if (pf) pf->begin(st);
  k_leaf_particular_rhs<T><<<grid_for(nl * rows * nrhs), 256, 0, st>>>(k, nl, nrhs, f, out, iti);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

__global__ void k_leaf_dtn_init_T(const double* QP, int nb, double s, int64_t nl, double* TH) {
  const int64_t per = (int64_t)nb * (nb + 1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * per;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int rc = (int)(e % per);
    TH[e] = (rc < nb * nb) ? s * QP[rc] : 0.0;
  }
}

cudaError_t leaf_dtn_init_T(const double* QP, int nb, double s, int64_t nl, double* TH,
                            cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_leaf_dtn_init_T<<<grid_for(nl * nb * (nb + 1)), 256, 0, st>>>(QP, nb, s, nl, TH);
  if (pf) pf->end(K_OTHER, 0.0, st);
  return cudaGetLastError();
}

// --------------------------------------------------------------- merges ----

__device__ inline void add_pair(double* p, double v) { atomicAdd(p, v); }
__device__ inline void add_pair(cplx* p, cplx v) {
  atomicAdd(&p->re, v.re);
  atomicAdd(&p->im, v.im);
}

// One thread per (merge, child, child row i, child column j <= nbc).
// DtN: D(var_i, var_j) += T (interface diagonal blocks get exactly two
// addends, so the result does not depend on their order); C and A entries
// and the h columns have a single owner except h_int, which also gets two.
// ItI: D(eq_i, var_j) = T on top of the identity, R(eq_i, .) = T, single owner.
template <typename T>
__global__ void k_merge_gather(const T* Tc, int64_t cstride, int nmerge, int nch, int nbc, int n_ext,
                               int n_int, const int* ext, const int* var, const int* eq, bool iti,
                               T* D, T* R, T* TP) {
  const int ncol = nbc + 1;
  const int64_t per_child = (int64_t)nbc * ncol;
  const int64_t total = (int64_t)nmerge * nch * per_child;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cidx = e / per_child;  // global child index = nch * merge + k
    const int rc = (int)(e % per_child);
    const int i = rc % nbc, j = rc / nbc;
    const int k = (int)(cidx % nch);
    const int64_t b = cidx / nch;
    const T v = Tc[cidx * cstride + rc];
    const int ei = ext[k * nbc + i];
    const int ri = iti ? eq[k * nbc + i] : var[k * nbc + i];
    T* Db = D + b * (int64_t)n_int * n_int;
    T* Rb = R + b * (int64_t)n_int * (n_ext + 1);
    T* Pb = TP + b * (int64_t)n_ext * (n_ext + 1);
    if (j == nbc) {  // h column
      if (ei >= 0) Pb[ei + (int64_t)n_ext * n_ext] = v;
      else if (iti) Rb[ri + (int64_t)n_int * n_ext] = v;
      else add_pair(&Rb[ri + (int64_t)n_int * n_ext], v);
      continue;
    }
    const int ej = ext[k * nbc + j];
    const int vj = var[k * nbc + j];
    if (ei >= 0) {
      if (ej >= 0) Pb[ei + (int64_t)ej * n_ext] = v;        // A
      // (exterior row, interior column) = B: used in place, not stored
    } else {
      if (ej >= 0) Rb[ri + (int64_t)ej * n_int] = v;         // C
      else if (iti) Db[ri + (int64_t)vj * n_int] = v;        // D12 / D21
      else add_pair(&Db[ri + (int64_t)vj * n_int], v);       // D
    }
  }
}

template <typename T>
cudaError_t merge_gather(const T* Tc, int64_t cstride, int nmerge, int nch, int nbc, int n_ext,
                         int n_int, const int* ext, const int* var, const int* eq, bool iti, T* D,
                         T* R, T* TP, cudaStream_t st, Prof* pf) {
  const int64_t total = (int64_t)nmerge * nch * nbc * (nbc + 1);
  if (pf) pf->begin(st);
  k_merge_gather<T><<<grid_for(total), 256, 0, st>>>(Tc, cstride, nmerge, nch, nbc, n_ext, n_int, ext,
                                                     var, eq, iti, D, R, TP);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_merge_gather_h(const T* hc, int nmerge, int nch, int nbc, int n_ext, int n_int,
                                 int nrhs, const int* ext, const int* var, const int* eq, bool iti,
                                 T* r, T* hp) {
  const int64_t per_child = (int64_t)nbc * nrhs;
  const int64_t total = (int64_t)nmerge * nch * per_child;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cidx = e / per_child;
    const int rc = (int)(e % per_child);
    const int i = rc % nbc, c = rc / nbc;
    const int k = (int)(cidx % nch);
    const int64_t b = cidx / nch;
    const T v = hc[cidx * per_child + rc];
    const int ei = ext[k * nbc + i];
    if (ei >= 0) {
      hp[b * (int64_t)n_ext * nrhs + ei + (int64_t)c * n_ext] = v;
    } else {
      const int ri = iti ? eq[k * nbc + i] : var[k * nbc + i];
      T* p = &r[b * (int64_t)n_int * nrhs + ri + (int64_t)c * n_int];
      if (iti) *p = v;
      else add_pair(p, v);
    }
  }
}

template <typename T>
cudaError_t merge_gather_h(const T* hc, int nmerge, int nch, int nbc, int n_ext, int n_int, int nrhs,
                           const int* ext, const int* var, const int* eq, bool iti, T* r, T* hp,
                           cudaStream_t st, Prof* pf) {
  const int64_t total = (int64_t)nmerge * nch * nbc * nrhs;
  if (pf) pf->begin(st);
  k_merge_gather_h<T><<<grid_for(total), 256, 0, st>>>(hc, nmerge, nch, nbc, n_ext, n_int, nrhs, ext,
                                                       var, eq, iti, r, hp);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

// ------------------------------------------------------------- downward ----

// gint(:, c) = -(X_C gpar(:, c) + xpart(:, c)); a warp per (merge, row, rhs)
// block of rows: each thread owns one row and walks the columns.
template <typename T>
__global__ void k_down_gint(const T* X, const T* xp, const T* gpar, int nmerge, int n_ext, int n_int,
                            int nrhs, T* gint) {
  const int64_t total = (int64_t)nmerge * n_int * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % n_int);
    const int64_t bc = e / n_int;
    const int c = (int)(bc % nrhs);
    const int64_t b = bc / nrhs;
    const T* Xb = X + b * (int64_t)n_int * (n_ext + 1);
    const T* g = gpar + b * (int64_t)n_ext * nrhs + (int64_t)c * n_ext;
    T acc = xp ? xp[b * (int64_t)n_int * nrhs + r + (int64_t)c * n_int] : Xb[r + (int64_t)n_ext * n_int];
    for (int j = 0; j < n_ext; ++j) acc = fmac(acc, Xb[r + (int64_t)j * n_int], g[j]);
    gint[b * (int64_t)n_int * nrhs + r + (int64_t)c * n_int] = -acc;
  }
}

// Same product for levels with few long rows (the top merges): a CTA holds
// 32 rows x CG column groups; each warp reads 32 consecutive rows of one
// column (coalesced), the CG partial sums are added in shared memory in a
// fixed order, so the result does not depend on scheduling.
template <typename T, int CG>
__global__ void __launch_bounds__(32 * CG) k_down_gint_split(const T* X, const T* xp, const T* gpar, int nmerge,
                                                         int n_ext, int n_int, int nrhs, T* gint) {
  __shared__ T part[CG][33];
  const int lane = threadIdx.x, cg = threadIdx.y;
  const int r = blockIdx.x * 32 + lane;
  const int64_t bc = blockIdx.y;  // merge * nrhs + rhs
  const int c = (int)(bc % nrhs);
  const int64_t b = bc / nrhs;
  const T* Xb = X + b * (int64_t)n_int * (n_ext + 1);
  const T* g = gpar + b * (int64_t)n_ext * nrhs + (int64_t)c * n_ext;
  T acc = T(0.0);
  if (r < n_int) {
    int j = cg;
#pragma unroll 4
    for (; j < n_ext; j += CG) acc = fmac(acc, Xb[r + (int64_t)j * n_int], g[j]);
  }
  part[cg][lane] = acc;
  __syncthreads();
  if (cg == 0 && r < n_int) {
    T s = xp ? xp[b * (int64_t)n_int * nrhs + r + (int64_t)c * n_int] : Xb[r + (int64_t)n_ext * n_int];
    for (int k = 0; k < CG; ++k) s = s + part[k][lane];
    gint[b * (int64_t)n_int * nrhs + r + (int64_t)c * n_int] = -s;
  }
}

// Rows of work below which the split kernel is used (about two resident
// threads per SM lane of the whole GPU would otherwise be idle).
constexpr int64_t kDownSplitRows = 1 << 17;

template <typename T>
void launch_down_gint(const T* X, const T* xp, const T* gpar, int nmerge, int n_ext, int n_int, int nrhs,
                      T* gint, cudaStream_t st) {
  const int64_t rows = (int64_t)nmerge * n_int * nrhs;
  if (rows < kDownSplitRows && n_ext >= 256 && (int64_t)nmerge * nrhs <= 65535) {
    dim3 grid((n_int + 31) / 32, nmerge * nrhs);
    k_down_gint_split<T, 16><<<grid, dim3(32, 16), 0, st>>>(X, xp, gpar, nmerge, n_ext, n_int, nrhs, gint);
  } else {
    k_down_gint<T><<<grid_for(rows, 128), 128, 0, st>>>(X, xp, gpar, nmerge, n_ext, n_int, nrhs, gint);
  }
}

template <typename T>
__global__ void k_down_children(const T* gpar, const T* gint, int nmerge, int nch, int nbc, int n_ext,
                                int n_int, int nrhs, const int* ext, const int* var, T* gchild) {
  const int64_t per_child = (int64_t)nbc * nrhs;
  const int64_t total = (int64_t)nmerge * nch * per_child;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cidx = e / per_child;
    const int rc = (int)(e % per_child);
    const int i = rc % nbc, c = rc / nbc;
    const int k = (int)(cidx % nch);
    const int64_t b = cidx / nch;
    const int ei = ext[k * nbc + i];
    T v;
    if (ei >= 0) v = gpar[b * (int64_t)n_ext * nrhs + ei + (int64_t)c * n_ext];
    else v = gint[b * (int64_t)n_int * nrhs + var[k * nbc + i] + (int64_t)c * n_int];
    gchild[e] = v;
  }
}

template <typename T>
cudaError_t down_level(const T* X, const T* xp, const T* gpar, int nmerge, int nch, int nbc, int n_ext,
                       int n_int, int nrhs, const int* ext, const int* var, T* gint, T* gchild,
                       cudaStream_t st, Prof* pf) {
  const double F = sizeof(T) == sizeof(cplx) ? 8.0 : 2.0;
  if (pf) pf->begin(st);
  launch_down_gint<T>(X, xp, gpar, nmerge, n_ext, n_int, nrhs, gint, st);
  if (pf) pf->end(K_DOWN, F * (double)nmerge * n_int * n_ext * nrhs, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (pf) pf->begin(st);
  k_down_children<T><<<grid_for((int64_t)nmerge * nch * nbc * nrhs), 256, 0, st>>>(
      gpar, gint, nmerge, nch, nbc, n_ext, n_int, nrhs, ext, var, gchild);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t down_gint(const T* X, const T* xp, const T* gpar, int nmerge, int n_ext, int n_int, int nrhs,
                      T* gint, cudaStream_t st, Prof* pf) {
  const double F = sizeof(T) == sizeof(cplx) ? 8.0 : 2.0;
  if (pf) pf->begin(st);
  launch_down_gint<T>(X, xp, gpar, nmerge, n_ext, n_int, nrhs, gint, st);
  if (pf) pf->end(K_DOWN, F * (double)nmerge * n_int * n_ext * nrhs, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t down_children(const T* gpar, const T* gint, int nmerge, int nch, int nbc, int n_ext, int n_int,
                          int nrhs, const int* ext, const int* var, T* gchild, cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_down_children<T><<<grid_for((int64_t)nmerge * nch * nbc * nrhs), 256, 0, st>>>(
      gpar, gint, nmerge, nch, nbc, n_ext, n_int, nrhs, ext, var, gchild);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_leaf_output(LeafConsts k, int64_t nl, int nrhs, const T* X, const T* xp, const T* g,
                              T* u, bool iti) {
  const int64_t total = (int64_t)nrhs * nl * k.npts;
  const int xrows = iti ? k.npts : k.ni;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int node = (int)(e % k.npts);
    const int64_t lc = e / k.npts;
    const int64_t leaf = lc % nl;
    const int c = (int)(lc / nl);
    const T* gl = g + (leaf * nrhs + c) * (int64_t)k.nb;
    const T* Xl = X + leaf * (int64_t)xrows * (k.nb + 1);
    T acc = T(0.0);
    if (iti) {
      acc = xp ? xp[(leaf * nrhs + c) * (int64_t)xrows + node] : Xl[node + (int64_t)k.nb * xrows];
      for (int j = 0; j < k.nb; ++j) acc = fmac(acc, Xl[node + (int64_t)j * xrows], gl[j]);
    } else {
      const int pr = k.prow[node];
      if (pr >= 0) {
        for (int j = 0; j < k.nb; ++j) acc = fmac(acc, T(k.P[pr + (int64_t)j * k.ne]), gl[j]);
      } else {
        const int r = k.iidx[node];
        acc = xp ? xp[(leaf * nrhs + c) * (int64_t)xrows + r] : Xl[r + (int64_t)k.nb * xrows];
        for (int j = 0; j < k.nb; ++j) acc = fmac(acc, Xl[r + (int64_t)j * xrows], gl[j]);
        acc = -acc;
      }
    }
    u[e] = acc;
  }
}

template <typename T>
cudaError_t leaf_output(const LeafConsts& k, int64_t nl, int nrhs, const T* X, const T* xp, const T* g,
                        T* u, bool iti, cudaStream_t st, Prof* pf) {
  const double F = sizeof(T) == sizeof(cplx) ? 8.0 : 2.0;
  if (pf) pf->begin(st);
  k_leaf_output<T><<<grid_for((int64_t)nrhs * nl * k.npts), 256, 0, st>>>(k, nl, nrhs, X, xp, g, u, iti);
  if (pf) pf->end(K_DOWN, F * (double)nrhs * nl * k.npts * k.nb, st);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_copy_block(const T* src, int64_t sstride, int sld, T* dst, int64_t dstride, int dld,
                             int m, int ncols, int batch) {
  const int64_t per = (int64_t)m * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * batch;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / per;
    const int rc = (int)(e % per);
    const int i = rc % m, j = rc / m;
    dst[b * dstride + i + (int64_t)j * dld] = src[b * sstride + i + (int64_t)j * sld];
  }
}

template <typename T>
cudaError_t copy_block(const T* src, int64_t sstride, int sld, T* dst, int64_t dstride, int dld, int m,
                       int ncols, int batch, cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_copy_block<T><<<grid_for((int64_t)m * ncols * batch), 256, 0, st>>>(src, sstride, sld, dst, dstride,
                                                                          dld, m, ncols, batch);
  if (pf) pf->end(K_OTHER, 0.0, st);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_scale_copy(const T* src, T* dst, int64_t n, double alpha) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = scale(src[e], alpha);
}

template <typename T>
cudaError_t scale_copy(const T* src, T* dst, int64_t n, double alpha, cudaStream_t st, Prof* pf) {
  if (pf) pf->begin(st);
  k_scale_copy<T><<<grid_for(n), 256, 0, st>>>(src, dst, n, alpha);
  if (pf) pf->end(K_OTHER, 0.0, st);
  return cudaGetLastError();
}

// ------------------------------------------------- grouped downward pass ----

// gint = -(X_C gpar + x) for one 32-row tile of one merge and right-hand
// side of one task per CTA: 32 lanes own the rows, 8 warps split the columns
// (coalesced 32-row column reads), partial sums added in shared memory in a
// fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_down_gint_group(DownGroup<T> grp) {
  __shared__ T part[8][33];
  const int lane = threadIdx.x, cg = threadIdx.y;
  const int64_t tile = blockIdx.x;
  int ti = 0;
  while (ti + 1 < grp.n && grp.t[ti + 1].tile0 <= tile) ++ti;
  const DownTask<T>& tk = grp.t[ti];
  const int rtiles = (tk.n_int + 31) / 32;
  const int64_t loc = tile - tk.tile0;
  const int r = (int)(loc % rtiles) * 32 + lane;
  const int64_t bc = loc / rtiles;
  const int c = (int)(bc % tk.nrhs);
  const int64_t b = bc / tk.nrhs;
  const T* Xb = tk.X + b * (int64_t)tk.n_int * (tk.n_ext + 1);
  const T* g = tk.gpar + b * (int64_t)tk.n_ext * tk.nrhs + (int64_t)c * tk.n_ext;
  T acc = T(0.0);
  if (r < tk.n_int) {
#pragma unroll 4
    for (int j = cg; j < tk.n_ext; j += 8) acc = fmac(acc, Xb[r + (int64_t)j * tk.n_int], g[j]);
  }
  part[cg][lane] = acc;
  __syncthreads();
  if (cg == 0 && r < tk.n_int) {
    T s = Xb[r + (int64_t)tk.n_ext * tk.n_int];
    for (int k = 0; k < 8; ++k) s = s + part[k][lane];
    tk.gint[b * (int64_t)tk.n_int * tk.nrhs + r + (int64_t)c * tk.n_int] = -s;
  }
}

template <typename T>
__global__ void k_down_children_group(DownGroup<T> grp) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < grp.elems;
       e += (int64_t)gridDim.x * blockDim.x) {
    int ti = 0;
    while (ti + 1 < grp.n && grp.t[ti + 1].elem0 <= e) ++ti;
    const DownTask<T>& tk = grp.t[ti];
    const int64_t le = e - tk.elem0;
    const int64_t per_child = (int64_t)tk.nbc * tk.nrhs;
    const int64_t cidx = le / per_child;
    const int rc = (int)(le % per_child);
    const int i = rc % tk.nbc, c = rc / tk.nbc;
    const int k = (int)(cidx % tk.nch);
    const int64_t b = cidx / tk.nch;
    const int ei = tk.ext[k * tk.nbc + i];
    T v;
    if (ei >= 0) v = tk.gpar[b * (int64_t)tk.n_ext * tk.nrhs + ei + (int64_t)c * tk.n_ext];
    else v = tk.gint[b * (int64_t)tk.n_int * tk.nrhs + tk.var[k * tk.nbc + i] + (int64_t)c * tk.n_int];
    tk.gchild[le] = v;
  }
}

template <typename T>
cudaError_t down_level_group(const DownGroup<T>& grp, cudaStream_t st) {
  if (grp.n <= 0) return cudaSuccess;
  if (grp.tiles > 0) k_down_gint_group<T><<<(unsigned)grp.tiles, dim3(32, 8), 0, st>>>(grp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (grp.elems > 0) k_down_children_group<T><<<grid_for(grp.elems), 256, 0, st>>>(grp);
  return cudaGetLastError();
}

// u = Y g + v with the build-time v, for the leaves of every task.
template <typename T>
__global__ void k_leaf_output_group(LeafGroup<T> grp) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < grp.elems;
       e += (int64_t)gridDim.x * blockDim.x) {
    int ti = 0;
    while (ti + 1 < grp.n && grp.t[ti + 1].elem0 <= e) ++ti;
    const LeafTask<T>& tk = grp.t[ti];
    const LeafConsts& k = tk.k;
    const int64_t le = e - tk.elem0;
    const int node = (int)(le % k.npts);
    const int64_t lc = le / k.npts;
    const int64_t leaf = lc % tk.nl;
    const int c = (int)(lc / tk.nl);
    const int xrows = grp.iti ? k.npts : k.ni;
    const T* gl = tk.g + (leaf * tk.nrhs + c) * (int64_t)k.nb;
    const T* Xl = tk.X + leaf * (int64_t)xrows * (k.nb + 1);
    T acc = T(0.0);
    if (grp.iti) {
      acc = Xl[node + (int64_t)k.nb * xrows];
      for (int j = 0; j < k.nb; ++j) acc = fmac(acc, Xl[node + (int64_t)j * xrows], gl[j]);
    } else {
      const int pr = k.prow[node];
      if (pr >= 0) {
        for (int j = 0; j < k.nb; ++j) acc = fmac(acc, T(k.P[pr + (int64_t)j * k.ne]), gl[j]);
      } else {
        const int r = k.iidx[node];
        acc = Xl[r + (int64_t)k.nb * xrows];
        for (int j = 0; j < k.nb; ++j) acc = fmac(acc, Xl[r + (int64_t)j * xrows], gl[j]);
        acc = -acc;
      }
    }
    tk.u[le] = acc;
  }
}

template <typename T>
cudaError_t leaf_output_group(const LeafGroup<T>& grp, cudaStream_t st) {
  if (grp.n <= 0 || grp.elems <= 0) return cudaSuccess;
  k_leaf_output_group<T><<<grid_for(grp.elems), 256, 0, st>>>(grp);
  return cudaGetLastError();
}

#define HPS_KINST(T)                                                                                  \
  template cudaError_t leaf_particular_rhs<T>(const LeafConsts&, int64_t, int, const T*, T*, bool,    \
                                              cudaStream_t, Prof*);                                   \
  template cudaError_t merge_gather<T>(const T*, int64_t, int, int, int, int, int, const int*,        \
                                       const int*, const int*, bool, T*, T*, T*, cudaStream_t, Prof*); \
  template cudaError_t merge_gather_h<T>(const T*, int, int, int, int, int, int, const int*,          \
                                         const int*, const int*, bool, T*, T*, cudaStream_t, Prof*);  \
  template cudaError_t down_level<T>(const T*, const T*, const T*, int, int, int, int, int, int,      \
                                     const int*, const int*, T*, T*, cudaStream_t, Prof*);            \
  template cudaError_t leaf_output<T>(const LeafConsts&, int64_t, int, const T*, const T*, const T*,  \
                                      T*, bool, cudaStream_t, Prof*);                                 \
  template cudaError_t copy_block<T>(const T*, int64_t, int, T*, int64_t, int, int, int, int,         \
                                     cudaStream_t, Prof*);                                            \
  template cudaError_t scale_copy<T>(const T*, T*, int64_t, double, cudaStream_t, Prof*);                 \
  template cudaError_t down_gint<T>(const T*, const T*, const T*, int, int, int, int, T*, cudaStream_t,     \
                                    Prof*);                                                                 \
  template cudaError_t down_children<T>(const T*, const T*, int, int, int, int, int, int, const int*,       \
                                        const int*, T*, cudaStream_t, Prof*);                                 \
  template cudaError_t down_level_group<T>(const DownGroup<T>&, cudaStream_t);                               \
  template cudaError_t leaf_output_group<T>(const LeafGroup<T>&, cudaStream_t);

HPS_KINST(double)
HPS_KINST(cplx)

}  // namespace hps
