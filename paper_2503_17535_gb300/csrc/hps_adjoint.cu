// Adjoint (conjugate-transposed) solve and coefficient gradients for uniform
// trees.  The HPS solve is a linear map (g, f) -> u: the leaf particular
// solves and h = Q v (Section 3.2), the upward merges x = D^{-1} h_int,
// h = h_ext - B x (Section 3.3, "merge outputs 1-2") and the downward pass
// g_int = -(X_C g + x), u = Y g + v (Section 3.4, Algorithm "down pass").
// hps_solve_adjoint applies the conjugate transpose of every step in reverse
// order with the stored factors, so (gbar, fbar) = (A_g^H ubar, A_f^H ubar).
// fbar is also the adjoint field of the collocation equations at the leaf
// interior nodes, from which hps_coeff_gradient forms the derivatives of
// Re<ubar, u> with respect to the coefficients a, b_k, c at those nodes.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "handle.h"

namespace hps {
namespace {

inline int gridn(int64_t total, int threads = 256) {
  int64_t b = (total + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 65535 * 8));
}

__device__ inline void atomic_add(double* p, double v) { atomicAdd(p, v); }
__device__ inline void atomic_add(cplx* p, cplx v) {
  atomicAdd(&p->re, v.re);
  atomicAdd(&p->im, v.im);
}
__device__ inline double re_of(double v) { return v; }
__device__ inline double re_of(cplx v) { return v.re; }

// gbar_leaf[leaf][j + c nb] = sum over nodes of d u[node] / d g[j] (conjugated) * ubar:
// ItI u = Y g + v: conj(Y)^T ubar; DtN u_bdry = P g, u_int = -(X_C g + x).
template <typename T>
__global__ void k_leaf_gbar(LeafConsts k, int64_t nl, int nrhs, const T* X, const T* ub, T* gleaf, bool iti) {
  const int64_t total = nl * nrhs * k.nb;
  const int xrows = iti ? k.npts : k.ni;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % k.nb);
    const int64_t lc = e / k.nb;
    const int c = (int)(lc % nrhs);
    const int64_t leaf = lc / nrhs;
    const T* u = ub + ((int64_t)c * nl + leaf) * k.npts;
    const T* Xl = X + leaf * (int64_t)xrows * (k.nb + 1) + (int64_t)j * xrows;
    T acc = T(0.0);
    if (iti) {
      for (int node = 0; node < k.npts; ++node) acc = fmac(acc, conj_of(Xl[node]), u[node]);
    } else {
      for (int node = 0; node < k.npts; ++node) {
        const int pr = k.prow[node];
        if (pr >= 0) acc = fmac(acc, T(k.P[pr + (int64_t)j * k.ne]), u[node]);
      }
      for (int r = 0; r < k.ni; ++r) acc = fmsc(acc, conj_of(Xl[r]), u[k.Ii[r]]);
    }
    gleaf[e] = acc;
  }
}

// xfbar[leaf][r + c xrows]: the v part of u (ItI: u = ... + v; DtN: u_int = ... - x).
template <typename T>
__global__ void k_leaf_xfbar(LeafConsts k, int64_t nl, int nrhs, const T* ub, T* xf, bool iti) {
  const int xrows = iti ? k.npts : k.ni;
  const int64_t total = nl * nrhs * xrows;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % xrows);
    const int64_t lc = e / xrows;
    const int c = (int)(lc % nrhs);
    const int64_t leaf = lc / nrhs;
    const T* u = ub + ((int64_t)c * nl + leaf) * k.npts;
    xf[e] = iti ? u[r] : -u[k.Ii[r]];
  }
}

// Transpose of k_down_children: every child boundary point's adjoint is
// added to the parent exterior entry or interior unknown it was copied from
// (gpar and gint zeroed before; at most two addends per entry, so the sums
// do not depend on their order).
template <typename T>
__global__ void k_down_children_adj(const T* gch, int nmerge, int nch, int nbc, int n_ext, int n_int, int nrhs,
                                    const int* ext, const int* var, T* gpar, T* gint) {
  const int64_t per_child = (int64_t)nbc * nrhs;
  const int64_t total = (int64_t)nmerge * nch * per_child;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cidx = e / per_child;
    const int rc = (int)(e % per_child);
    const int i = rc % nbc, c = rc / nbc;
    const int k = (int)(cidx % nch);
    const int64_t b = cidx / nch;
    const int ei = ext[k * nbc + i];
    const T v = gch[e];
    if (ei >= 0) atomic_add(&gpar[b * (int64_t)n_ext * nrhs + ei + (int64_t)c * n_ext], v);
    else atomic_add(&gint[b * (int64_t)n_int * nrhs + var[k * nbc + i] + (int64_t)c * n_int], v);
  }
}

// Transpose of k_merge_gather_h: each child point reads back the adjoint of
// the parent entry it was gathered into.
template <typename T>
__global__ void k_merge_gather_h_adj(const T* rbar, const T* hpbar, int nmerge, int nch, int nbc, int n_ext,
                                     int n_int, int nrhs, const int* ext, const int* var, const int* eq, bool iti,
                                     T* hcbar) {
  const int64_t per_child = (int64_t)nbc * nrhs;
  const int64_t total = (int64_t)nmerge * nch * per_child;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cidx = e / per_child;
    const int rc = (int)(e % per_child);
    const int i = rc % nbc, c = rc / nbc;
    const int k = (int)(cidx % nch);
    const int64_t b = cidx / nch;
    const int ei = ext[k * nbc + i];
    T v;
    if (ei >= 0) {
      v = hpbar ? hpbar[b * (int64_t)n_ext * nrhs + ei + (int64_t)c * n_ext] : T(0.0);
    } else {
      const int ri = iti ? eq[k * nbc + i] : var[k * nbc + i];
      v = rbar[b * (int64_t)n_int * nrhs + ri + (int64_t)c * n_int];
    }
    hcbar[e] = v;
  }
}

// Transpose of k_leaf_particular_rhs: fbar at the interior nodes (zero elsewhere).
template <typename T>
__global__ void k_particular_rhs_adj(LeafConsts k, int64_t nl, int nrhs, const T* tmp, T* fbar, bool iti) {
  const int rows = iti ? k.npts : k.ni;
  const int64_t total = nl * nrhs * k.ni;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % k.ni);
    const int64_t lc = e / k.ni;
    const int c = (int)(lc % nrhs);
    const int64_t leaf = lc / nrhs;
    const T v = tmp[leaf * (int64_t)rows * nrhs + (int64_t)c * rows + (iti ? k.nown + r : r)];
    fbar[((int64_t)c * nl + leaf) * k.npts + k.Ii[r]] = iti ? v : -v;
  }
}

// coefficient gradients at the interior nodes: -sum_c Re(conj(fbar) * (d/dcoef of L u))
template <typename T>
__global__ void k_coeff_grad(LeafConsts k, int64_t nl, int nrhs, const T* u, const T* fbar, double* ga, double* gb,
                             double* gc) {
  const int64_t total = nl * k.ni;
  const int p = k.p, dim = k.dim;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % k.ni);
    const int64_t leaf = e / k.ni;
    const int node = k.Ii[r];
    const int ix[3] = {node % p, (node / p) % p, dim == 3 ? node / (p * p) : 0};
    const int str[3] = {1, p, p * p};
    const double s = k.sleaf ? k.sleaf[leaf] : k.s;
    double sa = 0.0, sc = 0.0, sb[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < nrhs; ++c) {
      const T* ul = u + ((int64_t)c * nl + leaf) * k.npts;
      const T lam = conj_of(fbar[((int64_t)c * nl + leaf) * k.npts + node]);
      if (gc) sc -= re_of(lam * ul[node]);
      if (ga || gb) {
        T lap = T(0.0);
        for (int a = 0; a < dim; ++a) {
          const int base = node - ix[a] * str[a];
          T d1 = T(0.0), d2 = T(0.0);
          for (int m = 0; m < p; ++m) {
            const T v = ul[base + m * str[a]];
            d1 = fmac(d1, T(k.D[ix[a] * p + m]), v);
            d2 = fmac(d2, T(k.DD[ix[a] * p + m]), v);
          }
          lap = lap + scale(d2, s * s);
          sb[a] -= re_of(lam * scale(d1, s));
        }
        sa -= re_of(lam * lap);
      }
    }
    const int64_t o = leaf * k.npts + node;
    if (gc) gc[o] = sc;
    if (ga) ga[o] = sa;
    if (gb)
      for (int a = 0; a < dim; ++a) gb[(int64_t)a * nl * k.npts + o] = sb[a];
  }
}

// ---- host helpers

// The transpose of one child-block product of the ItI D route:
// forward C(eq) -= T_child(pts, pts) B(var); here Bbar(var) -= T^H Cbar(eq).
template <typename T>
cudaError_t child_block_h(hps_handle* h, int m, bool odd, BOp<T> Cbar, BOp<T> Bbar, int nrhs, cudaStream_t st,
                          Prof* pf) {
  LevelDev& Lv = h->lev[m];
  const int nb = h->nb;
  const T* Tcs = m == 0 ? (const T*)h->leafTH : (const T*)h->lev[m - 1].TP;
  const int64_t cst = m == 0 ? (int64_t)nb * (nb + 1) : (int64_t)h->lev[m - 1].n_ext * (h->lev[m - 1].n_ext + 1);
  const int hb = Lv.nbc / 2;
  GemmArgs<T> g;
  g.M = hb; g.N = nrhs; g.K = hb; g.batch = Lv.nmerge * 2;
  BOp<T> A = bop<T>(const_cast<T*>(Tcs) + (odd ? cst : 0), (int64_t)Lv.nch * cst, Lv.nbc);
  A.div = 2;
  A.sub = (odd ? 1 : 3) * cst;
  g.A = A;
  g.ta = true;
  g.arow.idx = odd ? Lv.odd_pts : Lv.even_pts; g.arow.len = hb; g.arow.period = 2;
  g.acol = g.arow;
  g.B = Cbar;
  g.brow.idx = odd ? Lv.odd_eq : Lv.even_eq; g.brow.len = hb; g.brow.period = 2;
  g.C = Bbar;
  g.crow.idx = odd ? Lv.odd_var : Lv.even_var; g.crow.len = hb; g.crow.period = 2;
  g.alpha = T(-1.0); g.beta = T(1.0);
  return gemm<T>(g, st, pf);
}

// b = D^{-H} y for every merge of level m (y overwritten; distinct buffers).
template <typename T>
hps_status apply_Dinv_h(hps_handle* h, int m, T* y, T* b, int nrhs, cudaStream_t st, Prof* pf) {
  LevelDev& Lv = h->lev[m];
  const int ni = Lv.n_int, nm = Lv.nmerge;
  BOp<T> YB = bop<T>(y, (int64_t)ni * nrhs, ni);
  BOp<T> BB = bop<T>(b, (int64_t)ni * nrhs, ni);
  if (!Kind<T>::iti) {
    HPS_CUDA(getrs_h<T>(bop<T>((T*)Lv.D, (int64_t)ni * ni, ni), ni, YB, nrhs, nm, st, pf));
    HPS_CUDA(permute_rows_inv<T>(YB, BB, Lv.perm, ni, nrhs, nm, st));
    return HPS_OK;
  }
  // forward: b1' = b1 - D12 b2; y1 = W^{-1} b1'; y2 = b2 - D21 y1
  const int hn = ni / 2;
  // y1bar += -D21^H y2bar  (forward D21 product: C = y rows even_eq, B = y rows even_var)
  HPS_CUDA(child_block_h<T>(h, m, false, grouped(YB, 2), grouped(YB, 2), nrhs, st, pf));
  // b2bar = y2bar
  HPS_CUDA(copy_block<T>(y + hn, (int64_t)ni * nrhs, ni, b + hn, (int64_t)ni * nrhs, ni, hn, nrhs, nm, st, pf));
  // b1'bar = W^{-H} y1bar
  HPS_CUDA(getrs_h<T>(bop<T>((T*)Lv.W, (int64_t)hn * hn, hn), hn, YB, nrhs, nm, st, pf));
  HPS_CUDA(permute_rows_inv<T>(YB, BB, Lv.perm, hn, nrhs, nm, st));
  // b2bar += -D12^H b1'bar  (forward D12 product: C = b rows odd_eq, B = b rows odd_var)
  HPS_CUDA(child_block_h<T>(h, m, true, grouped(BB, 2), grouped(BB, 2), nrhs, st, pf));
  return HPS_OK;
}

template <typename T>
hps_status adjoint_impl(hps_handle* h, int nrhs, const void* ub_in, void* gbar_out, void* fbar_out, cudaStream_t st) {
  constexpr bool ITI = Kind<T>::iti;
  HPS_TRY(ensure_solve_ws(h, nrhs));
  Prof* pf = &h->prof;
  pf->reset();
  pf->on = h->opts.profile != 0;
  const int64_t nl = h->nl;
  const int nb = h->nb, xr = h->xrows_leaf, nlu = h->nlu_leaf;
  const size_t ubytes = (size_t)nl * h->npts * nrhs * sizeof(T);
  // stage host buffers (ws_f holds ubar, ws_u receives fbar, ws_g gbar)
  const T* ub = (const T*)ub_in;
  if (!is_device_ptr(ub_in)) {
    HPS_CUDA(cudaMemcpyAsync(h->ws_f, ub_in, ubytes, cudaMemcpyHostToDevice, st));
    ub = (const T*)h->ws_f;
  }
  const bool host_g = gbar_out && !is_device_ptr(gbar_out);
  const bool host_f = fbar_out && !is_device_ptr(fbar_out);
  T* gbar = (!gbar_out || host_g) ? (T*)h->ws_g : (T*)gbar_out;
  T* fbar = (!fbar_out || host_f) ? (T*)h->ws_u : (T*)fbar_out;
  T* xf = (T*)h->ws_xf;     // xf bar, [leaf][xr x nrhs]
  T* tmp = (T*)h->ws_rhs;   // rhs bar
  T* gleaf = (T*)h->ws_gleaf;
  T* hleaf = (T*)h->ws_hleaf;
  const int L = h->L;

  // (5) leaf output: gbar_leaf = dY^H ubar, xfbar = v part
  k_leaf_gbar<T><<<gridn(nl * nrhs * nb), 256, 0, st>>>(h->lc, nl, nrhs, (const T*)h->leafX, ub, gleaf, ITI);
  HPS_CUDA(cudaGetLastError());
  k_leaf_xfbar<T><<<gridn(nl * nrhs * xr), 256, 0, st>>>(h->lc, nl, nrhs, ub, xf, ITI);
  HPS_CUDA(cudaGetLastError());

  // (4) downward pass, bottom-up: children's gbar -> parent gbar and gint bar;
  // xbar_m = -gint bar (lazy root: through D^{-H})
  const T* gch = gleaf;
  for (int m = 0; m < L; ++m) {
    LevelDev& Lv = h->lev[m];
    const int ne = Lv.n_ext, ni = Lv.n_int, nm = Lv.nmerge;
    T* gpar = (m == L - 1) ? gbar : (T*)h->lev[m + 1].gchild;
    T* gint = (T*)Lv.gint;
    HPS_CUDA(cudaMemsetAsync(gpar, 0, (size_t)nm * ne * nrhs * sizeof(T), st));
    HPS_CUDA(cudaMemsetAsync(gint, 0, (size_t)nm * ni * nrhs * sizeof(T), st));
    k_down_children_adj<T><<<gridn((int64_t)nm * Lv.nch * Lv.nbc * nrhs), 256, 0, st>>>(
        gch, nm, Lv.nch, Lv.nbc, ne, ni, nrhs, Lv.ext, Lv.var, gpar, gint);
    HPS_CUDA(cudaGetLastError());
    GemmArgs<T> g;
    g.M = ne; g.N = nrhs; g.K = ni; g.batch = nm;
    g.A = bop<T>((T*)Lv.X, (int64_t)ni * (ne + 1), ni);
    g.ta = true;
    g.B = bop<T>(gint, (int64_t)ni * nrhs, ni);
    g.C = bop<T>(gpar, (int64_t)ne * nrhs, ne);
    T* xb = (T*)Lv.x;
    if (Lv.lazy) {
      // forward: tmp = -(C g + r); gint = D^{-1} tmp.  tmpbar = D^{-H} gintbar
      HPS_TRY(apply_Dinv_h<T>(h, m, gint, xb, nrhs, st, pf));
      g.B = bop<T>(xb, (int64_t)ni * nrhs, ni);
      g.alpha = T(-1.0); g.beta = T(1.0);
      HPS_CUDA(gemm<T>(g, st, pf));
      // rbar = -tmpbar
      HPS_CUDA(scale_copy<T>(xb, (T*)Lv.r, (int64_t)nm * ni * nrhs, -1.0, st, pf));
    } else {
      g.alpha = T(-1.0); g.beta = T(1.0);
      HPS_CUDA(gemm<T>(g, st, pf));
      HPS_CUDA(scale_copy<T>(gint, xb, (int64_t)nm * ni * nrhs, -1.0, st, pf));
    }
    gch = gpar;
  }

  // (3) upward pass, top-down: xbar += -B^H hpbar; rbar = D^{-H} xbar;
  // children's hbar gathered back from rbar and hpbar
  for (int m = L - 1; m >= 0; --m) {
    LevelDev& Lv = h->lev[m];
    const int ne = Lv.n_ext, ni = Lv.n_int, nm = Lv.nmerge;
    T* xb = (T*)Lv.x;
    T* rb = (T*)Lv.r;
    const T* hpb = Lv.top() ? nullptr : (const T*)Lv.hp;
    if (!Lv.lazy) {
      if (!Lv.top()) {
        const T* Tc = m == 0 ? (const T*)h->leafTH : (const T*)h->lev[m - 1].TP;
        const int64_t cstride = m == 0 ? (int64_t)nb * (nb + 1) : (int64_t)h->lev[m - 1].n_ext * (h->lev[m - 1].n_ext + 1);
        const int hb = Lv.nbc / 2;
        if (ITI) {
          // each interior unknown belongs to one child: one product over all children
          GemmArgs<T> g;
          g.M = hb; g.N = nrhs; g.K = hb; g.batch = nm * Lv.nch;
          g.A = bop<T>(const_cast<T*>(Tc), cstride, Lv.nbc);
          g.ta = true;
          g.arow.idx = Lv.bacol; g.arow.len = hb; g.arow.period = Lv.nch;
          g.acol.idx = Lv.barow; g.acol.len = hb; g.acol.period = Lv.nch;
          g.B = grouped(bop<T>((T*)Lv.hp, (int64_t)ne * nrhs, ne), Lv.nch);
          g.brow.idx = Lv.bcrow; g.brow.len = hb; g.brow.period = Lv.nch;
          g.C = grouped(bop<T>(xb, (int64_t)ni * nrhs, ni), Lv.nch);
          g.crow.idx = Lv.bbrow; g.crow.len = hb; g.crow.period = Lv.nch;
          g.alpha = T(-1.0); g.beta = T(1.0);
          HPS_CUDA(gemm<T>(g, st, pf));
        } else {
          // DtN: an interface unknown is shared by two children, so the
          // products of neighbouring children must not run together
          const int half = Lv.nch / 2;
          for (int par = 0; par < 2; ++par) {
            if (!Lv.adj_ptrs[par]) {
              const MergeMaps mm = make_merge_maps(h->dim, Lv.n, false);
              std::vector<int> kids;
              for (int k2 = 0; k2 < Lv.nch; ++k2)
                if ((__builtin_popcount((unsigned)k2) & 1) == par) kids.push_back(k2);
              std::vector<T*> ptrs;
              for (int j = 0; j < nm; ++j)
                for (int k2 : kids) ptrs.push_back(const_cast<T*>(Tc) + ((int64_t)j * Lv.nch + k2) * cstride);
              std::vector<int> maps;
              for (const std::vector<int>* src : {&mm.b_arow, &mm.b_acol, &mm.b_brow, &mm.b_crow})
                for (int k2 : kids) maps.insert(maps.end(), src->begin() + (size_t)k2 * hb, src->begin() + (size_t)(k2 + 1) * hb);
              Lv.adj_ptrs[par] = upload(h, ptrs, st);
              Lv.adj_maps[par] = upload(h, maps, st);
              if (!Lv.adj_ptrs[par] || !Lv.adj_maps[par]) return HPS_ERR_OOM;
            }
            const int* mp = Lv.adj_maps[par];
            GemmArgs<T> g;
            g.M = hb; g.N = nrhs; g.K = hb; g.batch = nm * half;
            g.A = bopp<T>((T* const*)Lv.adj_ptrs[par], Lv.nbc);
            g.ta = true;
            g.arow.idx = mp + 1 * half * hb; g.arow.len = hb; g.arow.period = half;  // acol of the forward
            g.acol.idx = mp + 0 * half * hb; g.acol.len = hb; g.acol.period = half;  // arow of the forward
            BOp<T> HB = bop<T>((T*)Lv.hp, (int64_t)ne * nrhs, ne);
            HB.div = half;
            g.B = HB;
            g.brow.idx = mp + 3 * half * hb; g.brow.len = hb; g.brow.period = half;
            BOp<T> XB2 = bop<T>(xb, (int64_t)ni * nrhs, ni);
            XB2.div = half;
            g.C = XB2;
            g.crow.idx = mp + 2 * half * hb; g.crow.len = hb; g.crow.period = half;
            g.alpha = T(-1.0); g.beta = T(1.0);
            HPS_CUDA(gemm<T>(g, st, pf));
          }
        }
      }
      HPS_TRY(apply_Dinv_h<T>(h, m, xb, rb, nrhs, st, pf));
    }
    T* hcb = (m == 0) ? hleaf : (T*)h->lev[m - 1].hp;
    k_merge_gather_h_adj<T><<<gridn((int64_t)nm * Lv.nch * Lv.nbc * nrhs), 256, 0, st>>>(
        rb, hpb, nm, Lv.nch, Lv.nbc, ne, ni, nrhs, Lv.ext, Lv.var, Lv.eq, ITI, hcb);
    HPS_CUDA(cudaGetLastError());
  }
  if (L == 0) HPS_CUDA(cudaMemsetAsync(hleaf, 0, (size_t)nl * nb * nrhs * sizeof(T), st));

  // (2) leaf h = alpha * A_leaf xf: xfbar += conj(alpha) A_leaf^H hbar
  {
    GemmArgs<T> gl;
    gl.M = xr; gl.N = nrhs; gl.K = nb; gl.batch = (int)nl;
    gl.A = ITI ? bop<T>((T*)h->dQH, 0, nb) : bop<T>((T*)h->dQi, 0, nb);
    gl.ta = true;
    gl.B = bop<T>(hleaf, (int64_t)nb * nrhs, nb);
    gl.C = bop<T>(xf, (int64_t)xr * nrhs, xr);
    gl.alpha = ITI ? T(1.0) : T(-h->s);
    gl.beta = T(1.0);
    HPS_CUDA(gemm<T>(gl, st, pf));
  }
  // (1) leaf particular solves: tmpbar = P^T L^{-H} U^{-H} xfbar; fbar
  if (h->ie.on) {
    HPS_TRY(iti_elim_apply_h(h, (const cplx*)xf, (cplx*)tmp, nrhs, st, pf));
  } else {
    BOp<T> LA = bop<T>((T*)h->leafA, (int64_t)nlu * nlu, nlu);
    BOp<T> XF = bop<T>(xf, (int64_t)xr * nrhs, xr);
    HPS_CUDA(getrs_h<T>(LA, nlu, XF, nrhs, (int)nl, st, pf));
    HPS_CUDA(permute_rows_inv<T>(XF, bop<T>(tmp, (int64_t)xr * nrhs, xr), h->leaf_perm, nlu, nrhs, (int)nl, st));
  }
  HPS_CUDA(cudaMemsetAsync(fbar, 0, ubytes, st));
  k_particular_rhs_adj<T><<<gridn(nl * nrhs * h->lc.ni), 256, 0, st>>>(h->lc, nl, nrhs, tmp, fbar, ITI);
  HPS_CUDA(cudaGetLastError());
  if (host_g) HPS_CUDA(cudaMemcpyAsync(gbar_out, gbar, (size_t)h->nroot * nrhs * sizeof(T), cudaMemcpyDeviceToHost, st));
  if (host_f) HPS_CUDA(cudaMemcpyAsync(fbar_out, fbar, ubytes, cudaMemcpyDeviceToHost, st));
  if (host_g || host_f) HPS_CUDA(cudaStreamSynchronize(st));
  return HPS_OK;
}

}  // namespace

hps_status adjoint_solve(hps_handle* h, int nrhs, const void* ubar, void* gbar, void* fbar, cudaStream_t st) {
  if (!h || !ubar || nrhs < 1 || h->adaptive) return HPS_ERR_INVALID;
  return h->iti ? adjoint_impl<cplx>(h, nrhs, ubar, gbar, fbar, st)
                : adjoint_impl<double>(h, nrhs, ubar, gbar, fbar, st);
}

hps_status coeff_gradient(hps_handle* h, int nrhs, const void* u_in, const void* fb_in, double* ga, double* gb,
                          double* gc, cudaStream_t st) {
  if (!h || !u_in || !fb_in || nrhs < 1 || h->adaptive) return HPS_ERR_INVALID;
  if (!is_device_ptr(u_in) || !is_device_ptr(fb_in) || !is_device_ptr(ga) || !is_device_ptr(gb) ||
      !is_device_ptr(gc))
    return HPS_ERR_INVALID;
  const int64_t nl = h->nl;
  const int64_t n = nl * h->npts;
  for (double* g : {ga, gc})
    if (g) HPS_CUDA(cudaMemsetAsync(g, 0, (size_t)n * sizeof(double), st));
  if (gb) HPS_CUDA(cudaMemsetAsync(gb, 0, (size_t)n * h->dim * sizeof(double), st));
  if (h->iti)
    k_coeff_grad<cplx><<<gridn(nl * h->lc.ni), 256, 0, st>>>(h->lc, nl, nrhs, (const cplx*)u_in, (const cplx*)fb_in,
                                                           ga, gb, gc);
  else
    k_coeff_grad<double><<<gridn(nl * h->lc.ni), 256, 0, st>>>(h->lc, nl, nrhs, (const double*)u_in,
                                                             (const double*)fb_in, ga, gb, gc);
  HPS_CUDA(cudaGetLastError());
  return HPS_OK;
}

}  // namespace hps
