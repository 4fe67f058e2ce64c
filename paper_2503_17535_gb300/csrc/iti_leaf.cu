// ItI leaf solves by elimination of the interior nodes.
//
// Algorithm "2D ItI local solve" (Section 3.2, Appendix B.1) solves with the
// complex p^2 x p^2 matrix B = [G; L(I_i, :)].  Ordering its columns as
// boundary nodes (owner order) then interior nodes, and its rows as the
// impedance rows then the interior rows,
//     B = [[G_oe, G_oi], [L_ie, L_ii]],
// where only G_oe carries the complex i eta (on its diagonal) and the leaf
// operator blocks L_ie, L_ii are real (the coefficients are real).  Block
// elimination of the interior gives, for right-hand sides [r_o; r_i],
//     z   = L_ii^{-1} r_i                     (real factors, complex data)
//     y_e = S^{-1} (r_o - G_oi z),   S = G_oe - G_oi W,   W = L_ii^{-1} L_ie
//     y_i = z - W y_e,
// the same solution as B^{-1}, with the O(p^6) work in a real LU of the
// (p-2)^2 interior block instead of a complex LU of all p^2 nodes.  The
// interior block is the leaf's Dirichlet problem, so the path is taken only
// when that problem is far from resonance (checked by the caller from the
// coefficient bounds); otherwise the dense B route is used.
//
// Complex data against real factors is handled by splitting a complex
// n x m block into a real n x 2m block (real parts, then imaginary parts).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "handle.h"

namespace hps {
namespace {

inline int gridn(int64_t total, int threads = 256) {
  int64_t b = (total + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 65535 * 8));
}

// dst[leaf][r + c n] = Re / Im (c < m: real parts, c >= m: imaginary parts) of
// src[leaf][row(r) + c ld] (row(r) = rmap[r] or r0 + r); per-leaf strides.
__global__ void k_split(const cplx* src, int64_t sstride, int sld, const int* rmap, int r0, int n, int m,
                        int64_t nl, double* dst, int64_t dstride) {
  const int64_t per = (int64_t)n * 2 * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * per; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t leaf = e / per;
    const int rc = (int)(e % per);
    const int r = rc % n, c2 = rc / n;
    const int c = c2 % m;
    const int row = rmap ? rmap[r] : r0 + r;
    const cplx v = src[leaf * sstride + row + (int64_t)c * sld];
    dst[leaf * dstride + r + (int64_t)c2 * n] = c2 < m ? v.re : v.im;
  }
}

// dst[leaf][row(r) + c ld] = base[leaf][r + c bld] + sign * (re + i im) of the
// split block sp[leaf] (n x 2m); base may be null (0).
__global__ void k_merge(const double* sp, int64_t spstride, int n, int m, const cplx* base, int64_t bstride, int bld,
                        double sign, int64_t nl, cplx* dst, int64_t dstride, int dld, const int* rmap, int r0) {
  const int64_t per = (int64_t)n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * per; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t leaf = e / per;
    const int rc = (int)(e % per);
    const int r = rc % n, c = rc / n;
    const double* s = sp + leaf * spstride;
    cplx v(sign * s[r + (int64_t)c * n], sign * s[r + (int64_t)(m + c) * n]);
    if (base) v = v + base[leaf * bstride + r + (int64_t)c * bld];
    const int row = rmap ? rmap[r] : r0 + r;
    dst[leaf * dstride + row + (int64_t)c * dld] = v;
  }
}

// dst[leaf][row(r) + c ld] = src[leaf][r + c sld] (complex copy with a row map)
__global__ void k_copy_rows(const cplx* src, int64_t sstride, int sld, int n, int m, int64_t nl, cplx* dst,
                            int64_t dstride, int dld, const int* rmap, int r0, const int* smap) {
  const int64_t per = (int64_t)n * m;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * per; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t leaf = e / per;
    const int rc = (int)(e % per);
    const int r = rc % n, c = rc / n;
    const int srow = smap ? smap[r] : r;
    const int row = rmap ? rmap[r] : r0 + r;
    dst[leaf * dstride + row + (int64_t)c * dld] = src[leaf * sstride + srow + (int64_t)c * sld];
  }
}

// S[leaf] = complex(Sre[leaf]) + i eta on the diagonal
__global__ void k_make_S(const double* Sre, int no, double eta, int64_t nl, cplx* S) {
  const int64_t per = (int64_t)no * no;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * per; e += (int64_t)gridDim.x * blockDim.x) {
    const int rc = (int)(e % per);
    S[e] = cplx(Sre[e], (rc % no) == (rc / no) ? eta : 0.0);
  }
}

// dst[leaf] = src (shared) for every leaf
__global__ void k_broadcast(const double* src, int64_t n, int64_t nl, double* dst) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nl * n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e % n];
}

hps_status ensure_cap(hps_handle* h, int ncols) {
  ItiElim& E = h->ie;
  if (E.cap >= ncols) return HPS_OK;
  const int64_t nl = h->nl;
  const int cap = std::max(ncols, h->nb + 1);
  E.z = (double*)dalloc(h, (size_t)nl * E.ni * 2 * cap * sizeof(double));
  E.z2 = (double*)dalloc(h, (size_t)nl * E.ni * 2 * cap * sizeof(double));
  E.t = (double*)dalloc(h, (size_t)nl * E.no * 2 * cap * sizeof(double));
  E.q = (cplx*)dalloc(h, (size_t)nl * E.no * cap * sizeof(cplx));
  E.q2 = (cplx*)dalloc(h, (size_t)nl * E.no * cap * sizeof(cplx));
  if (!E.z || !E.z2 || !E.t || !E.q || !E.q2) return HPS_ERR_OOM;
  E.cap = cap;
  return HPS_OK;
}

}  // namespace

bool iti_elim_safe(hps_handle* h, const Coeffs& co, cudaStream_t st, hps_status* err) {
  *err = HPS_OK;
  if (h->opts.iti_leaf == 1) return false;
  if (h->opts.iti_leaf == 2) return true;
  double* d = (double*)dalloc(h, 192 * sizeof(double));
  if (!d) {
    *err = HPS_ERR_OOM;
    return false;
  }
  double b3[3];
  if (coef_bounds(co, h->dim, h->nl * h->npts, d, b3, st) != cudaSuccess) {
    cudaGetLastError();
    *err = HPS_ERR_CUDA;
    return false;
  }
  // first Dirichlet eigenvalue of -Lap on the leaf square, a = 1
  const double lam1 = 2.0 * M_PI * M_PI / (h->hlen * h->hlen);
  const double amin = b3[0], bmax = b3[1], cmax = b3[2];
  return amin > 0.0 && cmax <= 0.25 * amin * lam1 && bmax * h->hlen <= amin;
}

hps_status iti_elim_setup(hps_handle* h, const Coeffs& co, cudaStream_t st, Prof* pf) {
  ItiElim& E = h->ie;
  const ItiLeafRef& r = h->iref;
  const LeafConsts& k = h->lc;
  const int64_t nl = h->nl;
  const int p = h->p, ni = (int)r.Ii.size(), no = r.nown;
  E.on = true;
  E.ni = ni;
  E.no = no;
  // shared real parts of the impedance rows: sgn * s * d/dx_axis on the owner's line
  std::vector<double> Goe((size_t)no * no, 0.0), Goi((size_t)no * ni, 0.0);
  auto greal = [&](int row, int j) {
    const int node = r.own_node[row], ax = r.own_axis[row];
    const int ci[2] = {node % p, node / p}, cj[2] = {j % p, j / p};
    for (int a2 = 0; a2 < 2; ++a2)
      if (a2 != ax && ci[a2] != cj[a2]) return 0.0;
    return r.own_sgn[row] * h->s * h->spec.D[(size_t)ci[ax] * p + cj[ax]];
  };
  for (int row = 0; row < no; ++row) {
    for (int c = 0; c < no; ++c) Goe[(size_t)row + (size_t)c * no] = greal(row, r.own_node[c]);
    for (int c = 0; c < ni; ++c) Goi[(size_t)row + (size_t)c * no] = greal(row, r.Ii[c]);
  }
  E.Goe = upload(h, Goe, st);
  E.Goi = upload(h, Goi, st);
  E.LU = (double*)dalloc(h, (size_t)nl * ni * ni * sizeof(double));
  E.W = (double*)dalloc(h, (size_t)nl * ni * no * sizeof(double));
  E.S = (cplx*)dalloc(h, (size_t)nl * no * no * sizeof(cplx));
  E.ipiv = (int*)dalloc(h, (size_t)nl * ni * sizeof(int));
  E.perm = (int*)dalloc(h, (size_t)nl * ni * sizeof(int));
  E.ipivS = (int*)dalloc(h, (size_t)nl * no * sizeof(int));
  E.permS = (int*)dalloc(h, (size_t)nl * no * sizeof(int));
  if (!E.Goe || !E.Goi || !E.LU || !E.W || !E.S || !E.ipiv || !E.perm || !E.ipivS || !E.permS) return HPS_ERR_OOM;
  HPS_TRY(ensure_cap(h, h->nb + 1));
  // the build's scratch holds the temporaries (it is sized for nl x p^2 x (nb + 1) complex)
  double* tmp = (double*)h->scratch;
  HPS_CUDA(leaf_assemble_Lii(k, nl, co, E.LU, st, pf));
  HPS_CUDA(leaf_iti_Lie(k, nl, co, tmp, st, pf));
  E.G = lu_group_size<double>(ni, (int)std::min<int64_t>(nl, 1 << 30), h->num_sms);
  if (E.G > 1) {
    E.luw.bars = (unsigned*)dalloc(h, sizeof(unsigned) * 2 * nl);
    E.luw.pub_bytes = lu_pub_bytes<double>(ni, (int)nl, E.G);
    E.luw.pub = dalloc(h, E.luw.pub_bytes);
    if (!E.luw.bars || !E.luw.pub) return HPS_ERR_OOM;
    HPS_CUDA(cudaMemsetAsync(E.luw.bars, 0, sizeof(unsigned) * 2 * nl, st));
  }
  BOp<double> LUo = bop<double>(E.LU, (int64_t)ni * ni, ni);
  HPS_CUDA(getrf<double>(LUo, ni, (int)nl, E.ipiv, E.perm, h->leaf_info, h->dev_err, E.G, E.luw, st, pf));
  // W = L_ii^{-1} L_ie
  BOp<double> WB = bop<double>(E.W, (int64_t)ni * no, ni);
  HPS_CUDA(permute_rows<double>(bop<double>(tmp, (int64_t)ni * no, ni), WB, E.perm, ni, no, (int)nl, st, pf));
  HPS_CUDA(getrs_inplace<double>(LUo, ni, WB, no, (int)nl, st, pf));
  // S = G_oe - G_oi W (+ i eta on the diagonal)
  k_broadcast<<<gridn(nl * no * no), 256, 0, st>>>(E.Goe, (int64_t)no * no, nl, tmp);
  HPS_CUDA(cudaGetLastError());
  {
    GemmArgs<double> g;
    g.M = no; g.N = no; g.K = ni; g.batch = (int)nl;
    g.A = bop<double>(E.Goi, 0, no);
    g.B = WB;
    g.C = bop<double>(tmp, (int64_t)no * no, no);
    g.alpha = -1.0; g.beta = 1.0;
    HPS_CUDA(gemm<double>(g, st, pf));
  }
  k_make_S<<<gridn(nl * no * no), 256, 0, st>>>(tmp, no, h->eta, nl, E.S);
  HPS_CUDA(cudaGetLastError());
  E.GS = lu_group_size<cplx>(no, (int)std::min<int64_t>(nl, 1 << 30), h->num_sms);
  if (E.GS > 1) {
    E.luwS.bars = (unsigned*)dalloc(h, sizeof(unsigned) * 2 * nl);
    E.luwS.pub_bytes = lu_pub_bytes<cplx>(no, (int)nl, E.GS);
    E.luwS.pub = dalloc(h, E.luwS.pub_bytes);
    if (!E.luwS.bars || !E.luwS.pub) return HPS_ERR_OOM;
    HPS_CUDA(cudaMemsetAsync(E.luwS.bars, 0, sizeof(unsigned) * 2 * nl, st));
  }
  HPS_CUDA(getrf<cplx>(bop<cplx>(E.S, (int64_t)no * no, no), no, (int)nl, E.ipivS, E.permS, h->leaf_info, h->dev_err,
                       E.GS, E.luwS, st, pf));
  return HPS_OK;
}

// X = B^{-1} R for every leaf: R in the rows order of B ([impedance rows;
// interior rows], p^2 x m per leaf, leading dimension p^2), X in node order.
hps_status iti_elim_apply(hps_handle* h, const cplx* R, cplx* X, int m, cudaStream_t st, Prof* pf) {
  HPS_TRY(ensure_cap(h, m));
  ItiElim& E = h->ie;
  const int64_t nl = h->nl;
  const int ni = E.ni, no = E.no, xr = (int)h->npts;
  const int64_t xs = (int64_t)xr * m;
  // z = L_ii^{-1} r_i  (split into real / imaginary columns)
  k_split<<<gridn(nl * ni * 2 * m), 256, 0, st>>>(R, xs, xr, nullptr, no, ni, m, nl, E.z, (int64_t)ni * 2 * m);
  HPS_CUDA(cudaGetLastError());
  BOp<double> LUo = bop<double>(E.LU, (int64_t)ni * ni, ni);
  BOp<double> Z2 = bop<double>(E.z2, (int64_t)ni * 2 * m, ni);
  HPS_CUDA(permute_rows<double>(bop<double>(E.z, (int64_t)ni * 2 * m, ni), Z2, E.perm, ni, 2 * m, (int)nl, st, pf));
  HPS_CUDA(getrs_inplace<double>(LUo, ni, Z2, 2 * m, (int)nl, st, pf));
  // q = r_o - G_oi z
  {
    GemmArgs<double> g;
    g.M = no; g.N = 2 * m; g.K = ni; g.batch = (int)nl;
    g.A = bop<double>(E.Goi, 0, no);
    g.B = Z2;
    g.C = bop<double>(E.t, (int64_t)no * 2 * m, no);
    g.alpha = 1.0; g.beta = 0.0;
    HPS_CUDA(gemm<double>(g, st, pf));
  }
  k_merge<<<gridn(nl * no * m), 256, 0, st>>>(E.t, (int64_t)no * 2 * m, no, m, R, xs, xr, -1.0, nl, E.q,
                                              (int64_t)no * m, no, nullptr, 0);
  HPS_CUDA(cudaGetLastError());
  // y_e = S^{-1} q
  BOp<cplx> SB = bop<cplx>(E.S, (int64_t)no * no, no);
  BOp<cplx> Q2 = bop<cplx>(E.q2, (int64_t)no * m, no);
  HPS_CUDA(permute_rows<cplx>(bop<cplx>(E.q, (int64_t)no * m, no), Q2, E.permS, no, m, (int)nl, st, pf));
  HPS_CUDA(getrs_inplace<cplx>(SB, no, Q2, m, (int)nl, st, pf));
  // y_i = z - W y_e
  k_split<<<gridn(nl * no * 2 * m), 256, 0, st>>>(E.q2, (int64_t)no * m, no, nullptr, 0, no, m, nl, E.t,
                                                  (int64_t)no * 2 * m);
  HPS_CUDA(cudaGetLastError());
  {
    GemmArgs<double> g;
    g.M = ni; g.N = 2 * m; g.K = no; g.batch = (int)nl;
    g.A = bop<double>(E.W, (int64_t)ni * no, ni);
    g.B = bop<double>(E.t, (int64_t)no * 2 * m, no);
    g.C = Z2;
    g.alpha = -1.0; g.beta = 1.0;
    HPS_CUDA(gemm<double>(g, st, pf));
  }
  // scatter to node order
  k_copy_rows<<<gridn(nl * no * m), 256, 0, st>>>(E.q2, (int64_t)no * m, no, no, m, nl, X, xs, xr, h->downn, 0,
                                                  nullptr);
  HPS_CUDA(cudaGetLastError());
  k_merge<<<gridn(nl * ni * m), 256, 0, st>>>(E.z2, (int64_t)ni * 2 * m, ni, m, nullptr, 0, 0, 1.0, nl, X, xs, xr,
                                              h->dIi, 0);
  HPS_CUDA(cudaGetLastError());
  return HPS_OK;
}

// Rbar = B^{-H} Xbar: Xbar in node order, Rbar in the rows order of B.
//   x_o = S^{-H} (z_e - W^T z_i),  x_i = L_ii^{-T} (z_i - G_oi^T x_o)
hps_status iti_elim_apply_h(hps_handle* h, const cplx* Xb, cplx* Rb, int m, cudaStream_t st, Prof* pf) {
  HPS_TRY(ensure_cap(h, m));
  ItiElim& E = h->ie;
  const int64_t nl = h->nl;
  const int ni = E.ni, no = E.no, xr = (int)h->npts;
  const int64_t xs = (int64_t)xr * m;
  // z_e (complex, owner order) and z_i (split)
  k_copy_rows<<<gridn(nl * no * m), 256, 0, st>>>(Xb, xs, xr, no, m, nl, E.q, (int64_t)no * m, no, nullptr, 0,
                                                  h->downn);
  HPS_CUDA(cudaGetLastError());
  k_split<<<gridn(nl * ni * 2 * m), 256, 0, st>>>(Xb, xs, xr, h->dIi, 0, ni, m, nl, E.z, (int64_t)ni * 2 * m);
  HPS_CUDA(cudaGetLastError());
  // q = z_e - W^T z_i
  {
    GemmArgs<double> g;
    g.M = no; g.N = 2 * m; g.K = ni; g.batch = (int)nl;
    g.A = bop<double>(E.W, (int64_t)ni * no, ni);
    g.ta = true;
    g.B = bop<double>(E.z, (int64_t)ni * 2 * m, ni);
    g.C = bop<double>(E.t, (int64_t)no * 2 * m, no);
    g.alpha = 1.0; g.beta = 0.0;
    HPS_CUDA(gemm<double>(g, st, pf));
  }
  k_merge<<<gridn(nl * no * m), 256, 0, st>>>(E.t, (int64_t)no * 2 * m, no, m, E.q, (int64_t)no * m, no, -1.0, nl,
                                              E.q, (int64_t)no * m, no, nullptr, 0);
  HPS_CUDA(cudaGetLastError());
  // x_o = S^{-H} q
  BOp<cplx> QB = bop<cplx>(E.q, (int64_t)no * m, no);
  BOp<cplx> Q2 = bop<cplx>(E.q2, (int64_t)no * m, no);
  HPS_CUDA(getrs_h<cplx>(bop<cplx>(E.S, (int64_t)no * no, no), no, QB, m, (int)nl, st, pf));
  HPS_CUDA(permute_rows_inv<cplx>(QB, Q2, E.permS, no, m, (int)nl, st));
  // z_i -= G_oi^T x_o
  k_split<<<gridn(nl * no * 2 * m), 256, 0, st>>>(E.q2, (int64_t)no * m, no, nullptr, 0, no, m, nl, E.t,
                                                  (int64_t)no * 2 * m);
  HPS_CUDA(cudaGetLastError());
  BOp<double> ZB = bop<double>(E.z, (int64_t)ni * 2 * m, ni);
  {
    GemmArgs<double> g;
    g.M = ni; g.N = 2 * m; g.K = no; g.batch = (int)nl;
    g.A = bop<double>(E.Goi, 0, no);
    g.ta = true;
    g.B = bop<double>(E.t, (int64_t)no * 2 * m, no);
    g.C = ZB;
    g.alpha = -1.0; g.beta = 1.0;
    HPS_CUDA(gemm<double>(g, st, pf));
  }
  // x_i = L_ii^{-T} z_i
  BOp<double> Z2 = bop<double>(E.z2, (int64_t)ni * 2 * m, ni);
  HPS_CUDA(getrs_h<double>(bop<double>(E.LU, (int64_t)ni * ni, ni), ni, ZB, 2 * m, (int)nl, st, pf));
  HPS_CUDA(permute_rows_inv<double>(ZB, Z2, E.perm, ni, 2 * m, (int)nl, st));
  // Rbar rows: [x_o; x_i]
  k_copy_rows<<<gridn(nl * no * m), 256, 0, st>>>(E.q2, (int64_t)no * m, no, no, m, nl, Rb, xs, xr, nullptr, 0,
                                                  nullptr);
  HPS_CUDA(cudaGetLastError());
  k_merge<<<gridn(nl * ni * m), 256, 0, st>>>(E.z2, (int64_t)ni * 2 * m, ni, m, nullptr, 0, 0, 1.0, nl, Rb, xs, xr,
                                              nullptr, no);
  HPS_CUDA(cudaGetLastError());
  return HPS_OK;
}

}  // namespace hps
