// C ABI of the HPS solver: planning, storage, build (leaf stage + merges)
// and solve (upward particular pass, downward pass, leaf output).
#include <atomic>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "handle.h"
#include "hps_adaptive.h"

using namespace hps;

namespace {

hps_status check_tree(const hps_tree* t, int p, int q) {
  if (!t) return HPS_ERR_INVALID;
  if (t->dim != 2 && t->dim != 3) return HPS_ERR_INVALID;
  if (t->uniform_depth < 0 || t->morton || t->level) return HPS_ERR_INVALID;
  if (t->uniform_depth > (t->dim == 2 ? 12 : 7)) return HPS_ERR_INVALID;
  if (p < 4 || p > 24 || q != p - 2) return HPS_ERR_INVALID;
  const int64_t nl = (int64_t)1 << (t->dim * t->uniform_depth);
  if (t->n_leaves != nl) return HPS_ERR_INVALID;
  double side = t->hi[0] - t->lo[0];
  if (!(side > 0)) return HPS_ERR_INVALID;
  for (int a = 1; a < t->dim; ++a)
    if (!(std::fabs((t->hi[a] - t->lo[a]) - side) <= 1e-12 * side)) return HPS_ERR_INVALID;
  return HPS_OK;
}

int64_t nroot_of(int dim, int q, int L) {
  return dim == 2 ? 4LL * q * ((int64_t)1 << L) : 6LL * q * q * ((int64_t)1 << (2 * L));
}

// ------------------------------------------------------------- planning ----

template <typename T>
size_t plan_bytes(const hps_handle* h, bool with_solve_ws) {
  size_t b = 0;
  const size_t es = sizeof(T);
  const int64_t nl = h->nl;
  b += (size_t)nl * h->nlu_leaf * h->nlu_leaf * es;          // leaf LU
  b += (size_t)nl * h->xrows_leaf * (h->nb + 1) * es;        // leaf X
  b += (size_t)nl * h->nb * (h->nb + 1) * es;                // leaf T|h
  b += (size_t)nl * h->nlu_leaf * 3 * sizeof(int);
  size_t scratch = (size_t)nl * h->xrows_leaf * (h->nb + 1) * es;
  int n = h->n0 > 0 ? h->n0 : (h->dim == 2 ? h->q : h->q * h->q);
  int64_t nm = nl;
  for (int m = 0; m < h->L; ++m) {
    nm /= (h->dim == 2 ? 4 : 8);
    const int nf = 2 * h->dim;
    const int n_ext = nf * n * (h->dim == 2 ? 2 : 4);
    const int nif = h->dim == 2 ? 4 : 12;
    const int n_int = (h->iti ? 2 : 1) * nif * n;
    b += (size_t)nm * n_ext * (n_ext + 1) * es;   // TP
    b += (size_t)nm * n_int * n_int * es;         // D
    if (h->iti) b += (size_t)nm * (n_int / 2) * (n_int / 2) * es;
    b += (size_t)nm * n_int * (n_ext + 1) * es;   // X
    scratch = std::max(scratch, (size_t)nm * n_int * (n_ext + 1) * es);
    if (with_solve_ws) b += (size_t)nm * (3 * n_int + 2 * n_ext) * es * 2;
    n *= (h->dim == 2 ? 2 : 4);
  }
  b += scratch;
  return b;
}

// --------------------------------------------------------------- build -----

template <typename T>
hps_status build_impl(hps_handle* h, const hps_coeffs* cf, const void* f_in, cudaStream_t st) {
  constexpr bool ITI = Kind<T>::iti;
  const int dim = h->dim, p = h->p, q = h->q;
  Prof* pf = &h->prof;
  pf->reset();
  pf->on = h->opts.profile != 0;
  h->spec = make_spectral(p, q);
  h->s = 2.0 / h->hlen;
  if (!ITI) {
    h->dref = make_dtn_leaf(h->spec, dim);
    h->nb = h->dref.nb;
    h->nlu_leaf = h->dref.ni;
    h->xrows_leaf = h->dref.ni;
  } else {
    h->iref = make_iti_leaf(h->spec);
    h->nb = h->iref.nb;
    h->nlu_leaf = h->iref.npts;
    h->xrows_leaf = h->iref.npts;
  }
  if (h->ext_depth > 0) {
    // the leaves are subtree roots whose [T | h] the caller has put in leafTH
    const int side = 1 << h->ext_depth;
    h->nb = dim == 2 ? 4 * q * side : 6 * q * q * side * side;
    h->n0 = dim == 2 ? q * side : q * q * side * side;
    h->nlu_leaf = 0;
    h->xrows_leaf = 0;
  }
  // footprint check before any large allocation
  {
    size_t need = plan_bytes<T>(h, false) + ((size_t)64 << 20);
    size_t fr = 0, tot = 0;
    HPS_CUDA(cudaMemGetInfo(&fr, &tot));
    if (need > fr + dev_pool_idle_bytes()) return HPS_ERR_OOM;
  }
  // ---- constants
  h->dD = upload(h, h->spec.D, st);
  h->dDD = upload(h, h->spec.DD, st);
  std::vector<int> iidx(h->npts, -1);
  LeafConsts& k = h->lc;
  k.dim = dim; k.p = p; k.npts = (int)h->npts; k.nb = h->nb; k.s = h->s; k.eta = h->eta;
  k.D = h->dD; k.DD = h->dDD;
  if (!ITI) {
    const DtnLeafRef& r = h->dref;
    for (int i = 0; i < r.ni; ++i) iidx[r.Ii[i]] = i;
    h->dIi = upload(h, r.Ii, st);
    h->dprow = upload(h, r.prow, st);
    h->dP = upload(h, r.P, st);
    h->dQi = upload(h, r.Qi, st);
    h->dQP = upload(h, r.QP, st);
    k.ni = r.ni; k.ne = r.ne; k.nown = 0;
    k.Ii = h->dIi; k.prow = h->dprow; k.P = h->dP;
  } else {
    const ItiLeafRef& r = h->iref;
    for (size_t i = 0; i < r.Ii.size(); ++i) iidx[r.Ii[i]] = (int)i;
    h->dIi = upload(h, r.Ii, st);
    h->dP = upload(h, r.P, st);
    h->downn = upload(h, r.own_node, st);
    h->downa = upload(h, r.own_axis, st);
    h->dsgn = upload(h, r.own_sgn, st);
    std::vector<std::complex<double>> QH = make_iti_QH(h->spec, h->hlen, h->eta);
    std::vector<cplx> QHc(QH.size());
    for (size_t i = 0; i < QH.size(); ++i) QHc[i] = cplx(QH[i].real(), QH[i].imag());
    h->dQH = upload(h, QHc, st);
    std::vector<int> prow(h->npts, -1);
    h->dprow = upload(h, prow, st);
    k.ni = (int)r.Ii.size(); k.ne = 0; k.nown = r.nown;
    k.Ii = h->dIi; k.prow = h->dprow; k.P = h->dP;
    k.own_node = h->downn; k.own_axis = h->downa; k.own_sgn = h->dsgn;
  }
  h->diidx = upload(h, iidx, st);
  k.iidx = h->diidx;
  if (!h->dD || !h->dDD || !h->dIi || !h->dP || !h->diidx || !h->dprow) return HPS_ERR_OOM;
  if (!ITI && (!h->dQi || !h->dQP)) return HPS_ERR_OOM;
  if (ITI && (!h->downn || !h->downa || !h->dsgn || !h->dQH)) return HPS_ERR_OOM;
  h->dev_err = (unsigned*)dalloc(h, sizeof(unsigned) * 4);
  if (!h->dev_err) return HPS_ERR_OOM;
  HPS_CUDA(cudaMemsetAsync(h->dev_err, 0, sizeof(unsigned) * 4, st));

  // ---- input staging (coefficients and f may live in host memory)
  std::vector<void*> tmp;
  auto stage = [&](const void* src, size_t bytes) -> const void* {
    if (!src || is_device_ptr(src)) return src;
    void* d = dalloc(h, bytes, &tmp);
    if (!d) return nullptr;
    if (cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return nullptr;
    return d;
  };
  const size_t cbytes = (size_t)h->nl * h->npts * sizeof(double);
  Coeffs co{};
  co.a = (const double*)stage(cf->a, cbytes);
  for (int a = 0; a < 3; ++a) co.b[a] = (a < dim) ? (const double*)stage(cf->b[a], cbytes) : nullptr;
  co.c = (const double*)stage(cf->c, cbytes);
  const T* f = (const T*)stage(f_in, (size_t)h->nl * h->npts * sizeof(T));
  if ((cf->a && !co.a) || (cf->c && !co.c) || (f_in && !f)) return HPS_ERR_OOM;
  for (int a = 0; a < dim; ++a)
    if (cf->b[a] && !co.b[a]) return HPS_ERR_OOM;

  // ---- leaf stage (Algorithm "local solve")
  const int64_t nl = h->nl;
  const int nlu = h->nlu_leaf, nb = h->nb, xr = h->xrows_leaf;
  const bool ext = h->ext_depth > 0;
  bool elim = false;
  if (ITI && !ext) {
    hps_status es = HPS_OK;
    elim = iti_elim_safe(h, co, st, &es);
    if (es != HPS_OK) return es;
  }
  if (!elim && !ext) {
    h->leafA = dalloc(h, (size_t)nl * nlu * nlu * sizeof(T));
    h->leaf_ipiv = (int*)dalloc(h, (size_t)nl * nlu * sizeof(int));
    h->leaf_perm = (int*)dalloc(h, (size_t)nl * nlu * sizeof(int));
    if (!h->leafA || !h->leaf_ipiv || !h->leaf_perm) return HPS_ERR_OOM;
  }
  if (!ext) {
    h->leafX = dalloc(h, (size_t)nl * xr * (nb + 1) * sizeof(T));
    h->leafTH = dalloc(h, (size_t)nl * nb * (nb + 1) * sizeof(T));
  }
  h->leaf_info = (int*)dalloc(h, (size_t)nl * sizeof(int));
  // scratch: largest R / RHS buffer of any stage
  size_t scratch = (size_t)nl * xr * (nb + 1);
  {
    int n = h->n0 > 0 ? h->n0 : (dim == 2 ? q : q * q);
    int64_t nm = nl;
    for (int m = 0; m < h->L; ++m) {
      nm /= (dim == 2 ? 4 : 8);
      MergeMaps mm = make_merge_maps(dim, n, ITI);
      scratch = std::max(scratch, (size_t)nm * mm.n_int * (mm.n_ext + 1));
      n *= (dim == 2 ? 2 : 4);
    }
  }
  h->scratch = dalloc(h, std::max<size_t>(scratch, 1) * sizeof(T));
  if ((!ext && !h->leafX) || !h->leafTH || !h->leaf_info || !h->scratch) return HPS_ERR_OOM;
  HPS_CUDA(cudaMemsetAsync(h->leaf_info, 0, (size_t)nl * sizeof(int), st));
  T* RHS = (T*)h->scratch;
  BOp<T> LX = bop<T>((T*)h->leafX, (int64_t)xr * (nb + 1), xr);
  if (ext) {
    // nothing to do at the leaves
  } else if (elim) {
    // ItI by elimination of the interior nodes: X = B^{-1} [[P, 0], [0, f_i]]
    HPS_TRY(iti_elim_setup(h, co, st, pf));
    HPS_CUDA(leaf_iti_rhs(k, nl, (const cplx*)f, (cplx*)RHS, st, pf));
    HPS_TRY(iti_elim_apply(h, (const cplx*)RHS, (cplx*)h->leafX, nb + 1, st, pf));
  } else if (!ITI) {
    HPS_CUDA(leaf_dtn_assemble(k, nl, co, (const double*)f, (double*)h->leafA, (double*)RHS, st, pf));
  } else {
    HPS_CUDA(leaf_iti_assemble(k, nl, co, (const cplx*)f, (cplx*)h->leafA, (cplx*)RHS, st, pf));
  }
  if (!elim && !ext) {
    h->leaf_G = lu_group_size<T>(nlu, (int)std::min<int64_t>(nl, 1 << 30), h->num_sms);
    if (h->leaf_G > 1) {
      h->leaf_luw.bars = (unsigned*)dalloc(h, sizeof(unsigned) * 2 * nl);
      h->leaf_luw.pub_bytes = lu_pub_bytes<T>(nlu, (int)nl, h->leaf_G);
      h->leaf_luw.pub = dalloc(h, h->leaf_luw.pub_bytes);
      if (!h->leaf_luw.bars || !h->leaf_luw.pub) return HPS_ERR_OOM;
      HPS_CUDA(cudaMemsetAsync(h->leaf_luw.bars, 0, sizeof(unsigned) * 2 * nl, st));
    }
    BOp<T> LA = bop<T>((T*)h->leafA, (int64_t)nlu * nlu, nlu);
    HPS_CUDA(getrf<T>(LA, nlu, (int)nl, h->leaf_ipiv, h->leaf_perm, h->leaf_info, h->dev_err, h->leaf_G,
                      h->leaf_luw, st, pf));
    HPS_CUDA(permute_rows<T>(bop<T>(RHS, (int64_t)xr * (nb + 1), xr), LX, h->leaf_perm, nlu, nb + 1, (int)nl, st, pf));
    HPS_CUDA(getrs_inplace<T>(LA, nlu, LX, nb + 1, (int)nl, st, pf));
  }
  if (!ext) {
    GemmArgs<T> g;
    g.M = nb; g.N = nb + 1; g.batch = (int)nl;
    g.B = LX;
    g.C = bop<T>((T*)h->leafTH, (int64_t)nb * (nb + 1), nb);
    if (!ITI) {
      HPS_CUDA(leaf_dtn_init_T(h->dQP, nb, h->s, nl, (double*)h->leafTH, st, pf));
      g.K = xr;
      g.A = bop<T>((T*)h->dQi, 0, nb);
      g.alpha = T(-h->s);
      g.beta = T(1.0);
    } else {
      g.K = (int)h->npts;
      g.A = bop<T>((T*)h->dQH, 0, nb);
      g.alpha = T(1.0);
      g.beta = T(0.0);
    }
    HPS_CUDA(gemm<T>(g, st, pf));
  }

  // ---- merge stage (Algorithm "merge"), level by level
  int n = h->n0 > 0 ? h->n0 : (dim == 2 ? q : q * q);
  int64_t nm = nl;
  const T* Tc = (const T*)h->leafTH;
  int64_t cstride = (int64_t)nb * (nb + 1);
  h->lev.resize(h->L);
  for (int m = 0; m < h->L; ++m) {
    LevelDev& Lv = h->lev[m];
    const int nch = dim == 2 ? 4 : 8;
    nm /= nch;
    MergeMaps mm = make_merge_maps(dim, n, ITI);
    Lv.nmerge = (int)nm; Lv.nch = nch; Lv.n = n; Lv.nbc = mm.nbc; Lv.n_ext = mm.n_ext; Lv.n_int = mm.n_int;
    Lv.ext = upload(h, mm.ext, st);
    Lv.var = upload(h, mm.var, st);
    Lv.eq = upload(h, mm.eq, st);
    Lv.barow = upload(h, mm.b_arow, st);
    Lv.bacol = upload(h, mm.b_acol, st);
    Lv.bbrow = upload(h, mm.b_brow, st);
    Lv.bcrow = upload(h, mm.b_crow, st);
    if (ITI) {
      const int hb = mm.nbc / 2;
      auto pick = [&](int c0, int c1, const std::vector<int>& src) {
        std::vector<int> v(src.begin() + (size_t)c0 * hb, src.begin() + (size_t)(c0 + 1) * hb);
        v.insert(v.end(), src.begin() + (size_t)c1 * hb, src.begin() + (size_t)(c1 + 1) * hb);
        return v;
      };
      Lv.odd_pts = upload(h, pick(1, 2, mm.b_acol), st);
      Lv.odd_var = upload(h, pick(1, 2, mm.b_brow), st);
      Lv.odd_eq = upload(h, pick(1, 2, mm.i_eq), st);
      Lv.even_pts = upload(h, pick(0, 3, mm.b_acol), st);
      Lv.even_var = upload(h, pick(0, 3, mm.b_brow), st);
      Lv.even_eq = upload(h, pick(0, 3, mm.i_eq), st);
      if (!Lv.odd_pts || !Lv.odd_var || !Lv.odd_eq || !Lv.even_pts || !Lv.even_var || !Lv.even_eq)
        return HPS_ERR_OOM;
    }
    const int ne = mm.n_ext, ni = mm.n_int;
    const int nlu_m = ITI ? ni / 2 : ni;
    Lv.TP = dalloc(h, (size_t)nm * ne * (ne + 1) * sizeof(T));
    Lv.D = dalloc(h, (size_t)nm * ni * ni * sizeof(T));
    if (ITI) Lv.W = dalloc(h, (size_t)nm * nlu_m * nlu_m * sizeof(T));
    Lv.X = dalloc(h, (size_t)nm * ni * (ne + 1) * sizeof(T));
    Lv.ipiv = (int*)dalloc(h, (size_t)nm * nlu_m * sizeof(int));
    Lv.perm = (int*)dalloc(h, (size_t)nm * nlu_m * sizeof(int));
    Lv.info = (int*)dalloc(h, (size_t)nm * sizeof(int));
    if (!Lv.ext || !Lv.var || !Lv.eq || !Lv.barow || !Lv.bacol || !Lv.bbrow || !Lv.bcrow || !Lv.TP ||
        !Lv.D || (ITI && !Lv.W) || !Lv.X || !Lv.ipiv || !Lv.perm || !Lv.info)
      return HPS_ERR_OOM;
    HPS_CUDA(cudaMemsetAsync(Lv.info, 0, (size_t)nm * sizeof(int), st));
    Lv.lazy = Lv.top() && h->opts.lazy_root && !h->opts.want_root_map;
    if (Lv.lazy && nm == 1) {
      // flags and a host-mapped error word for the flag-ordered solves
      const int nf = (ni + 31) / 32;
      h->trsv.flags = (unsigned*)dalloc(h, (size_t)nf * sizeof(unsigned));
      h->trsv.dinv = dalloc(h, (size_t)2 * nf * 1024 * sizeof(T));
      h->trsv.dinv_ready = false;
      if (!h->trsv.flags || !h->trsv.dinv) return HPS_ERR_OOM;
      HPS_CUDA(cudaMemsetAsync(h->trsv.flags, 0, (size_t)nf * sizeof(unsigned), st));
      h->trsv.nflags = nf;
      HPS_CUDA(cudaHostAlloc((void**)&h->trsv_err_host, sizeof(int), cudaHostAllocMapped));
      *h->trsv_err_host = 0;
      int* dp = nullptr;
      HPS_CUDA(cudaHostGetDevicePointer((void**)&dp, h->trsv_err_host, 0));
      h->trsv.host_err = h->trsv_err_host;
      h->trsv.dev_err = dp;
    }
    // at a lazy root [C | h_int] is kept (in X's storage) instead of X
    T* R = Lv.lazy ? (T*)Lv.X : (T*)h->scratch;
    // D, R = [C | h_int], TP = [A | h_ext]
    HPS_CUDA(fill<T>(bop<T>((T*)Lv.D, (int64_t)ni * ni, ni), ni, ni, (int)nm, T(0.0), ITI ? T(1.0) : T(0.0), st, pf));
    HPS_CUDA(fill<T>(bop<T>(R, (int64_t)ni * (ne + 1), ni), ni, ne + 1, (int)nm, T(0.0), T(0.0), st, pf));
    HPS_CUDA(fill<T>(bop<T>((T*)Lv.TP, (int64_t)ne * (ne + 1), ne), ne, ne + 1, (int)nm, T(0.0), T(0.0), st, pf));
    HPS_CUDA(merge_gather<T>(Tc, cstride, (int)nm, nch, mm.nbc, ne, ni, Lv.ext, Lv.var, Lv.eq, ITI,
                             (T*)Lv.D, R, (T*)Lv.TP, st, pf));
    Lv.G = lu_group_size<T>(nlu_m, (int)nm, h->num_sms);
    if (Lv.G > 1) {
      Lv.luw.bars = (unsigned*)dalloc(h, sizeof(unsigned) * 2 * nm);
      Lv.luw.pub_bytes = lu_pub_bytes<T>(nlu_m, (int)nm, Lv.G);
      Lv.luw.pub = dalloc(h, Lv.luw.pub_bytes);
      if (!Lv.luw.bars || !Lv.luw.pub) return HPS_ERR_OOM;
      HPS_CUDA(cudaMemsetAsync(Lv.luw.bars, 0, sizeof(unsigned) * 2 * nm, st));
    }
    BOp<T> XX = bop<T>((T*)Lv.X, (int64_t)ni * (ne + 1), ni);
    if (!ITI) {
      BOp<T> DD = bop<T>((T*)Lv.D, (int64_t)ni * ni, ni);
      HPS_CUDA(getrf<T>(DD, ni, (int)nm, Lv.ipiv, Lv.perm, Lv.info, h->dev_err, Lv.G, Lv.luw, st, pf));
      if (!Lv.lazy) {
        HPS_CUDA(permute_rows<T>(bop<T>(R, (int64_t)ni * (ne + 1), ni), XX, Lv.perm, ni, ne + 1, (int)nm, st, pf));
        HPS_CUDA(getrs_inplace<T>(DD, ni, XX, ne + 1, (int)nm, st, pf));
      }
    } else {
      const int hn = ni / 2;
      BOp<T> D12 = bop<T>((T*)Lv.D, (int64_t)ni * ni, ni, (int64_t)hn * ni);
      BOp<T> D21 = bop<T>((T*)Lv.D, (int64_t)ni * ni, ni, (int64_t)hn);
      BOp<T> WW = bop<T>((T*)Lv.W, (int64_t)hn * hn, hn);
      BOp<T> R1 = bop<T>(R, (int64_t)ni * (ne + 1), ni);
      BOp<T> R2 = bop<T>(R, (int64_t)ni * (ne + 1), ni, hn);
      (void)D12;
      (void)R2;
      // D12 (D21) is nonzero only in the interior-interior blocks of the odd
      // (even) children: its product with a matrix is one gathered product
      // per child, rows = the child's equation rows, K = its interior points.
      const int hb = mm.nbc / 2;
      auto child_block = [&](bool odd, BOp<T> B, BOp<T> C, int N) {
        GemmArgs<T> g;
        g.M = hb; g.N = N; g.K = hb; g.batch = (int)nm * 2;
        BOp<T> A = bop<T>(const_cast<T*>(Tc) + (odd ? cstride : 0), (int64_t)nch * cstride, mm.nbc);
        A.div = 2;
        A.sub = (odd ? 1 : 3) * cstride;
        g.A = A;
        g.arow.idx = odd ? Lv.odd_pts : Lv.even_pts; g.arow.len = hb; g.arow.period = 2;
        g.acol = g.arow;
        g.B = B;
        g.brow.idx = odd ? Lv.odd_var : Lv.even_var; g.brow.len = hb; g.brow.period = 2;
        g.C = C;
        g.crow.idx = odd ? Lv.odd_eq : Lv.even_eq; g.crow.len = hb; g.crow.period = 2;
        g.alpha = T(-1.0); g.beta = T(1.0);
        return gemm<T>(g, st, pf);
      };
      // W = I - D12 D21 (Eq. "ItI D inverse"): rows of the odd children's
      // equations, D21 read from D's lower-left block (rows = own vars)
      HPS_CUDA(fill<T>(WW, hn, hn, (int)nm, T(0.0), T(1.0), st, pf));
      HPS_CUDA(child_block(true, grouped(bop<T>((T*)Lv.D, (int64_t)ni * ni, ni), 2), grouped(WW, 2), hn));
      if (Lv.lazy) {
        HPS_CUDA(getrf<T>(WW, hn, (int)nm, Lv.ipiv, Lv.perm, Lv.info, h->dev_err, Lv.G, Lv.luw, st, pf));
        goto merged;
      }
      // R1 <- R1 - D12 R2
      HPS_CUDA(child_block(true, grouped(bop<T>(R, (int64_t)ni * (ne + 1), ni), 2),
                           grouped(bop<T>(R, (int64_t)ni * (ne + 1), ni), 2), ne + 1));
      HPS_CUDA(getrf<T>(WW, hn, (int)nm, Lv.ipiv, Lv.perm, Lv.info, h->dev_err, Lv.G, Lv.luw, st, pf));
      // X1 = W^{-1} R1
      HPS_CUDA(permute_rows<T>(R1, XX, Lv.perm, hn, ne + 1, (int)nm, st, pf));
      HPS_CUDA(getrs_inplace<T>(WW, hn, XX, ne + 1, (int)nm, st, pf));
      // X2 = R2 - D21 X1
      HPS_CUDA(copy_block<T>(R + hn, (int64_t)ni * (ne + 1), ni, (T*)Lv.X + hn, (int64_t)ni * (ne + 1), ni, hn,
                             ne + 1, (int)nm, st, pf));
      (void)D21;
      HPS_CUDA(child_block(false, grouped(XX, 2), grouped(XX, 2), ne + 1));
    }
  merged:
    // [T | h] = [A | h_ext] - B X  (block-sparse: one product per child)
    if (!Lv.top() || h->opts.want_root_map) {
      GemmArgs<T> g;
      g.M = mm.nbc / 2; g.N = ne + 1; g.K = mm.nbc / 2; g.batch = (int)(nm * nch);
      g.A = bop<T>(const_cast<T*>(Tc), cstride, mm.nbc);
      g.arow.idx = Lv.barow; g.arow.len = mm.nbc / 2; g.arow.period = nch;
      g.acol.idx = Lv.bacol; g.acol.len = mm.nbc / 2; g.acol.period = nch;
      g.B = grouped(bop<T>((T*)Lv.X, (int64_t)ni * (ne + 1), ni), nch);
      g.brow.idx = Lv.bbrow; g.brow.len = mm.nbc / 2; g.brow.period = nch;
      g.C = grouped(bop<T>((T*)Lv.TP, (int64_t)ne * (ne + 1), ne), nch);
      g.crow.idx = Lv.bcrow; g.crow.len = mm.nbc / 2; g.crow.period = nch;
      g.alpha = T(-1.0); g.beta = T(1.0);
      HPS_CUDA(gemm<T>(g, st, pf));
    }
    Tc = (const T*)Lv.TP;
    cstride = (int64_t)ne * (ne + 1);
    n *= (dim == 2 ? 2 : 4);
  }

  // ---- status: singular pivots / timeouts
  HPS_CUDA(cudaStreamSynchronize(st));
  for (void* t : tmp) { dev_free(t, st); }
  unsigned derr = 0;
  HPS_CUDA(cudaMemcpy(&derr, h->dev_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (derr & DEV_ERR_TIMEOUT) return HPS_ERR_TIMEOUT;
  {
    std::vector<int> info(nl);
    HPS_CUDA(cudaMemcpy(info.data(), h->leaf_info, nl * sizeof(int), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < nl; ++i)
      if (info[i]) { h->err_node = i; return HPS_ERR_SINGULAR; }
    int64_t off = nl;
    for (int m = 0; m < h->L; ++m) {
      std::vector<int> li(h->lev[m].nmerge);
      HPS_CUDA(cudaMemcpy(li.data(), h->lev[m].info, li.size() * sizeof(int), cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < li.size(); ++i)
        if (li[i]) { h->err_node = off + (int64_t)i; return HPS_ERR_SINGULAR; }
      off += h->lev[m].nmerge;
    }
  }
  return HPS_OK;
}

// --------------------------------------------------------------- solve -----

void drop_graphs(hps_handle* h);

template <typename T>
hps_status ensure_ws(hps_handle* h, int nrhs) {
  if (h->ws_nrhs >= nrhs) return HPS_OK;
  if (h->capturing) return HPS_ERR_INVALID;  // never allocate inside a capture
  drop_graphs(h);                            // they refer to the old buffers
  // the call has ordered h->last after the handle's earlier work
  for (void* pp : h->ws_allocs) { dev_free(pp, h->last); }
  h->ws_allocs.clear();
  h->bytes -= h->ws_bytes;
  const int64_t before = h->bytes;
  h->ws_nrhs = 0;
  const size_t es = sizeof(T);
  auto A = [&](size_t bytes) { return dalloc(h, bytes, &h->ws_allocs); };
  h->ws_xf = A((size_t)h->nl * h->xrows_leaf * nrhs * es);
  h->ws_hleaf = A((size_t)h->nl * h->nb * nrhs * es);
  h->ws_gleaf = A((size_t)h->nl * h->nb * nrhs * es);
  h->ws_g = A((size_t)h->nroot * nrhs * es);
  h->ws_f = A((size_t)h->nl * h->npts * nrhs * es);
  h->ws_u = A((size_t)h->nl * h->npts * nrhs * es);
  h->ws_rhs = A((size_t)h->nl * h->xrows_leaf * nrhs * es);
  if (!h->ws_xf || !h->ws_hleaf || !h->ws_gleaf || !h->ws_g || !h->ws_f || !h->ws_u || !h->ws_rhs)
    return HPS_ERR_OOM;
  for (int m = 0; m < h->L; ++m) {
    LevelDev& Lv = h->lev[m];
    const int64_t nm = Lv.nmerge;
    Lv.r = A((size_t)nm * Lv.n_int * nrhs * es);
    Lv.x = A((size_t)nm * Lv.n_int * nrhs * es);
    Lv.hp = A((size_t)nm * Lv.n_ext * nrhs * es);
    Lv.gint = A((size_t)nm * Lv.n_int * nrhs * es);
    Lv.gchild = A((size_t)nm * Lv.nch * Lv.nbc * nrhs * es);
    if (!Lv.r || !Lv.x || !Lv.hp || !Lv.gint || !Lv.gchild) return HPS_ERR_OOM;
  }
  h->ws_bytes = h->bytes - before;
  h->ws_nrhs = nrhs;
  return HPS_OK;
}

// y = D^{-1} b for every merge of level m and nrhs columns (b, y: n_int x
// nrhs per merge, column-major, distinct buffers; b is overwritten).  DtN:
// the LU factors of D.  ItI: D = [[I, D12], [D21, I]] with W = I - D12 D21
// factored; D12 / D21 blocks are read from the children's T (block-sparse).
template <typename T>
hps_status apply_Dinv(hps_handle* h, int m, T* b, T* y, int nrhs, cudaStream_t st, Prof* pf) {
  LevelDev& Lv = h->lev[m];
  const int ni = Lv.n_int, nm = Lv.nmerge;
  BOp<T> YB = bop<T>(y, (int64_t)ni * nrhs, ni);
  if (!Kind<T>::iti) {
    BOp<T> DD = bop<T>((T*)Lv.D, (int64_t)ni * ni, ni);
    HPS_CUDA(permute_rows<T>(bop<T>(b, (int64_t)ni * nrhs, ni), YB, Lv.perm, ni, nrhs, nm, st, pf));
    if (!h->capturing && trsv_flags_applicable<T>(ni, nrhs, nm, h->trsv))
      HPS_CUDA(getrs_flags<T>((const T*)Lv.D, ni, ni, y, ni, nrhs, h->trsv, st, pf));
    else
      HPS_CUDA(getrs_inplace<T>(DD, ni, YB, nrhs, nm, st, pf));
    return HPS_OK;
  }
  const int hn = ni / 2, nb = h->nb;
  BOp<T> WW = bop<T>((T*)Lv.W, (int64_t)hn * hn, hn);
  BOp<T> B1 = bop<T>(b, (int64_t)ni * nrhs, ni);
  const T* Tcs = m == 0 ? (const T*)h->leafTH : (const T*)h->lev[m - 1].TP;
  const int64_t cst = m == 0 ? (int64_t)nb * (nb + 1) : (int64_t)h->lev[m - 1].n_ext * (h->lev[m - 1].n_ext + 1);
  const int hb = Lv.nbc / 2;
  auto child_block = [&](bool odd, BOp<T> B, BOp<T> C) {
    GemmArgs<T> g;
    g.M = hb; g.N = nrhs; g.K = hb; g.batch = nm * 2;
    BOp<T> A = bop<T>(const_cast<T*>(Tcs) + (odd ? cst : 0), (int64_t)Lv.nch * cst, Lv.nbc);
    A.div = 2;
    A.sub = (odd ? 1 : 3) * cst;
    g.A = A;
    g.arow.idx = odd ? Lv.odd_pts : Lv.even_pts; g.arow.len = hb; g.arow.period = 2;
    g.acol = g.arow;
    g.B = B;
    g.brow.idx = odd ? Lv.odd_var : Lv.even_var; g.brow.len = hb; g.brow.period = 2;
    g.C = C;
    g.crow.idx = odd ? Lv.odd_eq : Lv.even_eq; g.crow.len = hb; g.crow.period = 2;
    g.alpha = T(-1.0); g.beta = T(1.0);
    return gemm<T>(g, st, pf);
  };
  // b1 <- b1 - D12 b2 (odd children's interior blocks)
  HPS_CUDA(child_block(true, grouped(B1, 2), grouped(B1, 2)));
  HPS_CUDA(permute_rows<T>(B1, YB, Lv.perm, hn, nrhs, nm, st, pf));
  if (!h->capturing && trsv_flags_applicable<T>(hn, nrhs, nm, h->trsv))
    HPS_CUDA(getrs_flags<T>((const T*)Lv.W, hn, hn, y, ni, nrhs, h->trsv, st, pf));
  else
    HPS_CUDA(getrs_inplace<T>(WW, hn, YB, nrhs, nm, st, pf));
  HPS_CUDA(copy_block<T>(b + hn, (int64_t)ni * nrhs, ni, y + hn, (int64_t)ni * nrhs, ni, hn, nrhs, nm, st, pf));
  // y2 <- b2 - D21 y1 (even children's interior blocks)
  HPS_CUDA(child_block(false, grouped(YB, 2), grouped(YB, 2)));
  return HPS_OK;
}

template <typename T>
hps_status solve_impl(hps_handle* h, int nrhs, const void* g_in, const void* f_in, void* u_out,
                      cudaStream_t st) {
  constexpr bool ITI = Kind<T>::iti;
  // a bounded wait of an earlier flag-ordered solve on this handle gave up
  if (h->trsv_err_host && *(volatile int*)h->trsv_err_host) return HPS_ERR_TIMEOUT;
  hps_status rs = ensure_ws<T>(h, nrhs);
  if (rs != HPS_OK) return rs;
  Prof* pf = &h->prof;
  pf->reset();
  pf->on = h->opts.profile != 0;
  const int64_t nl = h->nl;
  const int nb = h->nb, xr = h->xrows_leaf, nlu = h->nlu_leaf;
  // stage host inputs
  // (a captured solve has checked its pointers before the capture began)
  const T* g = (const T*)g_in;
  if (!h->capturing && !is_device_ptr(g_in)) {
    HPS_CUDA(cudaMemcpyAsync(h->ws_g, g_in, (size_t)h->nroot * nrhs * sizeof(T), cudaMemcpyHostToDevice, st));
    g = (const T*)h->ws_g;
  }
  const T* f = (const T*)f_in;
  if (f_in && !h->capturing && !is_device_ptr(f_in)) {
    HPS_CUDA(cudaMemcpyAsync(h->ws_f, f_in, (size_t)nl * h->npts * nrhs * sizeof(T), cudaMemcpyHostToDevice, st));
    f = (const T*)h->ws_f;
  }
  const bool ext = h->ext_depth > 0;  // leaves are subtree roots: no leaf solves, no leaf output
  const bool host_u = !ext && !h->capturing && !is_device_ptr(u_out);
  T* u = host_u ? (T*)h->ws_u : (T*)u_out;
  const bool newf = (f != nullptr) || (ext && h->ext_newf);

  // ---- upward particular pass (new f): leaf and merge triangular solves
  if (newf && !ext) {
    T* xf = (T*)h->ws_xf;
    T* tmp = (T*)h->ws_rhs;
    HPS_CUDA(leaf_particular_rhs<T>(h->lc, nl, nrhs, f, tmp, ITI, st, pf));
    BOp<T> XF = bop<T>(xf, (int64_t)xr * nrhs, xr);
    if (h->ie.on) {
      HPS_TRY(iti_elim_apply(h, (const cplx*)tmp, (cplx*)xf, nrhs, st, pf));
    } else {
      BOp<T> LA = bop<T>((T*)h->leafA, (int64_t)nlu * nlu, nlu);
      HPS_CUDA(permute_rows<T>(bop<T>(tmp, (int64_t)xr * nrhs, xr), XF, h->leaf_perm, nlu, nrhs, (int)nl, st, pf));
      HPS_CUDA(getrs_inplace<T>(LA, nlu, XF, nrhs, (int)nl, st, pf));
    }
    GemmArgs<T> gl;
    gl.M = nb; gl.N = nrhs; gl.K = ITI ? (int)h->npts : xr; gl.batch = (int)nl;
    gl.A = ITI ? bop<T>((T*)h->dQH, 0, nb) : bop<T>((T*)h->dQi, 0, nb);
    gl.B = XF;
    gl.C = bop<T>((T*)h->ws_hleaf, (int64_t)nb * nrhs, nb);
    gl.alpha = ITI ? T(1.0) : T(-h->s);
    gl.beta = T(0.0);
    HPS_CUDA(gemm<T>(gl, st, pf));
  }
  if (newf) {
    // leaves' h (for subtree roots: put in ws_hleaf by the caller)
    const T* hc = (const T*)h->ws_hleaf;
    for (int m = 0; m < h->L; ++m) {
      LevelDev& Lv = h->lev[m];
      const int ne = Lv.n_ext, ni = Lv.n_int, nm = Lv.nmerge;
      T* r = (T*)Lv.r;
      T* x = (T*)Lv.x;
      HPS_CUDA(fill<T>(bop<T>(r, (int64_t)ni * nrhs, ni), ni, nrhs, nm, T(0.0), T(0.0), st, pf));
      HPS_CUDA(merge_gather_h<T>(hc, nm, Lv.nch, Lv.nbc, ne, ni, nrhs, Lv.ext, Lv.var, Lv.eq, ITI, r,
                                 (T*)Lv.hp, st, pf));
      if (Lv.lazy) break;  // the root's D^{-1} is applied in the downward pass
      HPS_TRY(apply_Dinv<T>(h, m, r, x, nrhs, st, pf));
      if (!Lv.top()) {
        GemmArgs<T> g;
        g.M = Lv.nbc / 2; g.N = nrhs; g.K = Lv.nbc / 2; g.batch = nm * Lv.nch;
        const T* Tc = m == 0 ? (const T*)h->leafTH : (const T*)h->lev[m - 1].TP;
        const int64_t cstride = m == 0 ? (int64_t)nb * (nb + 1)
                                       : (int64_t)h->lev[m - 1].n_ext * (h->lev[m - 1].n_ext + 1);
        g.A = bop<T>(const_cast<T*>(Tc), cstride, Lv.nbc);
        g.arow.idx = Lv.barow; g.arow.len = Lv.nbc / 2; g.arow.period = Lv.nch;
        g.acol.idx = Lv.bacol; g.acol.len = Lv.nbc / 2; g.acol.period = Lv.nch;
        g.B = grouped(bop<T>(x, (int64_t)ni * nrhs, ni), Lv.nch);
        g.brow.idx = Lv.bbrow; g.brow.len = Lv.nbc / 2; g.brow.period = Lv.nch;
        g.C = grouped(bop<T>((T*)Lv.hp, (int64_t)ne * nrhs, ne), Lv.nch);
        g.crow.idx = Lv.bcrow; g.crow.len = Lv.nbc / 2; g.crow.period = Lv.nch;
        g.alpha = T(-1.0); g.beta = T(1.0);
        HPS_CUDA(gemm<T>(g, st, pf));
      }
      hc = (const T*)Lv.hp;
    }
  }

  // ---- downward pass (Algorithm "down pass")
  const T* gpar = g;
  for (int m = h->L - 1; m >= 0; --m) {
    LevelDev& Lv = h->lev[m];
    T* gchild = (m == 0) ? (T*)h->ws_gleaf : (T*)Lv.gchild;
    if (Lv.lazy) {
      // Lv.X = [C | h_int]: t = -(C g + h), with the solve's own h when f is new,
      // then g_int = D^{-1} t
      HPS_CUDA(down_gint<T>((const T*)Lv.X, newf ? (const T*)Lv.r : nullptr, gpar, Lv.nmerge, Lv.n_ext,
                            Lv.n_int, nrhs, (T*)Lv.x, st, pf));
      HPS_TRY(apply_Dinv<T>(h, m, (T*)Lv.x, (T*)Lv.gint, nrhs, st, pf));
      HPS_CUDA(down_children<T>(gpar, (const T*)Lv.gint, Lv.nmerge, Lv.nch, Lv.nbc, Lv.n_ext, Lv.n_int, nrhs,
                                Lv.ext, Lv.var, gchild, st, pf));
    } else {
      HPS_CUDA(down_level<T>((const T*)Lv.X, newf ? (const T*)Lv.x : nullptr, gpar, Lv.nmerge, Lv.nch,
                             Lv.nbc, Lv.n_ext, Lv.n_int, nrhs, Lv.ext, Lv.var, (T*)Lv.gint, gchild, st, pf));
    }
    gpar = gchild;
  }
  // leaf output u = Y g + v (subtree roots: their g stays in ws_gleaf)
  if (ext) return HPS_OK;
  HPS_CUDA(leaf_output<T>(h->lc, nl, nrhs, (const T*)h->leafX, newf ? (const T*)h->ws_xf : nullptr, gpar, u,
                          ITI, st, pf));
  if (host_u) {
    HPS_CUDA(cudaMemcpyAsync(u_out, u, (size_t)nl * h->npts * nrhs * sizeof(T), cudaMemcpyDeviceToHost, st));
    HPS_CUDA(cudaStreamSynchronize(st));
    if (h->trsv_err_host && *(volatile int*)h->trsv_err_host) return HPS_ERR_TIMEOUT;
  }
  return HPS_OK;
}

// Apply-only solves (build-time source) of several operators, the same
// level of every tree in one launch (Section 3.4, Algorithm "down pass", for
// many trees at once): per level counted from the roots one grouped gint
// launch and one grouped children launch, then one grouped leaf output.  A
// lazy root is applied per operator first (its D^{-1} is a factored solve).
template <typename T>
hps_status solve_multi_impl(const std::vector<int>& idx, hps_handle* const* hs, const int* nrhs,
                            const void* const* g, void* const* u, cudaStream_t st) {
  int maxL = 0;
  for (int i : idx) {
    hps_handle* h = hs[i];
    if (h->trsv_err_host && *(volatile int*)h->trsv_err_host) return HPS_ERR_TIMEOUT;
    HPS_TRY(ensure_ws<T>(h, nrhs[i]));
    maxL = std::max(maxL, h->L);
    if (h->L > 0 && h->lev[h->L - 1].lazy) {
      LevelDev& Lv = h->lev[h->L - 1];
      T* gchild = (h->L == 1) ? (T*)h->ws_gleaf : (T*)Lv.gchild;
      HPS_CUDA(down_gint<T>((const T*)Lv.X, nullptr, (const T*)g[i], Lv.nmerge, Lv.n_ext, Lv.n_int, nrhs[i],
                            (T*)Lv.x, st, nullptr));
      HPS_TRY(apply_Dinv<T>(h, h->L - 1, (T*)Lv.x, (T*)Lv.gint, nrhs[i], st, nullptr));
      HPS_CUDA(down_children<T>((const T*)g[i], (const T*)Lv.gint, Lv.nmerge, Lv.nch, Lv.nbc, Lv.n_ext, Lv.n_int,
                                nrhs[i], Lv.ext, Lv.var, gchild, st, nullptr));
    }
  }
  DownGroup<T> grp;
  auto flush_down = [&]() -> cudaError_t {
    cudaError_t e = down_level_group<T>(grp, st);
    grp.n = 0;
    grp.tiles = grp.elems = 0;
    return e;
  };
  for (int d = 0; d < maxL; ++d) {
    grp.n = 0;
    grp.tiles = grp.elems = 0;
    for (int i : idx) {
      hps_handle* h = hs[i];
      if (h->L <= d) continue;
      const int m = h->L - 1 - d;
      LevelDev& Lv = h->lev[m];
      if (d == 0 && Lv.lazy) continue;
      DownTask<T>& tk = grp.t[grp.n++];
      tk.X = (const T*)Lv.X;
      tk.gpar = d == 0 ? (const T*)g[i] : (const T*)h->lev[m + 1].gchild;
      tk.gint = (T*)Lv.gint;
      tk.gchild = m == 0 ? (T*)h->ws_gleaf : (T*)Lv.gchild;
      tk.ext = Lv.ext;
      tk.var = Lv.var;
      tk.nmerge = Lv.nmerge; tk.nch = Lv.nch; tk.nbc = Lv.nbc;
      tk.n_ext = Lv.n_ext; tk.n_int = Lv.n_int; tk.nrhs = nrhs[i];
      tk.tile0 = grp.tiles;
      tk.elem0 = grp.elems;
      grp.tiles += (int64_t)Lv.nmerge * ((Lv.n_int + 31) / 32) * nrhs[i];
      grp.elems += (int64_t)Lv.nmerge * Lv.nch * Lv.nbc * nrhs[i];
      if (grp.n == kMaxGroup) HPS_CUDA(flush_down());
    }
    HPS_CUDA(flush_down());
  }
  LeafGroup<T> lg;
  lg.n = 0;
  lg.iti = Kind<T>::iti;
  lg.elems = 0;
  for (int i : idx) {
    hps_handle* h = hs[i];
    LeafTask<T>& tk = lg.t[lg.n++];
    tk.k = h->lc;
    tk.nl = h->nl;
    tk.nrhs = nrhs[i];
    tk.X = (const T*)h->leafX;
    tk.g = h->L > 0 ? (const T*)h->ws_gleaf : (const T*)g[i];
    tk.u = (T*)u[i];
    tk.elem0 = lg.elems;
    lg.elems += (int64_t)nrhs[i] * h->nl * h->npts;
    if (lg.n == kMaxGroup) {
      HPS_CUDA(leaf_output_group<T>(lg, st));
      lg.n = 0;
      lg.elems = 0;
    }
  }
  HPS_CUDA(leaf_output_group<T>(lg, st));
  return HPS_OK;
}

// ------------------------------------------------ subtree recomputation ----

void handle_begin(hps_handle* h, cudaStream_t st);
void handle_end(hps_handle* h, cudaStream_t st);
//
// Paper Section 4.1, Algorithm "our_recomputation", on the device only: the
// tree below level L - d is cut into its complete subtrees of depth d (the
// largest d whose peak footprint fits the budget, as the paper picks the
// largest subtrees that fit).  The build runs each subtree's leaf stage and
// merges to its root, keeps only the root's T and h, and releases the rest;
// the merges above the subtree roots are kept as usual.  A solve runs the
// upward pass above the roots (new sources: each subtree is rebuilt with the
// new source to get its root's h), the downward pass to the roots, then
// rebuilds each subtree and runs its own downward pass and leaf output.  A
// subtree's leaves are a contiguous range of leaves (Morton order), so its
// coefficients, sources and solutions are slices of the caller's arrays.

namespace {

int64_t uniform_plan(int dim, int depth, int p, int q, bool iti, int ext_depth, bool with_ws) {
  hps_handle t;
  t.dim = dim; t.p = p; t.q = q; t.L = depth; t.iti = iti;
  t.nl = (int64_t)1 << (dim * depth);
  t.npts = dim == 2 ? (int64_t)p * p : (int64_t)p * p * p;
  const int64_t ni = dim == 2 ? (int64_t)(p - 2) * (p - 2) : (int64_t)(p - 2) * (p - 2) * (p - 2);
  t.nb = dim == 2 ? 4 * q : 6 * q * q;
  t.nlu_leaf = (int)(iti ? t.npts : ni);
  t.xrows_leaf = t.nlu_leaf;
  if (ext_depth > 0) {
    const int side = 1 << ext_depth;
    t.nb = dim == 2 ? 4 * q * side : 6 * q * q * side * side;
    t.n0 = dim == 2 ? q * side : q * q * side * side;
    t.nlu_leaf = 0;
    t.xrows_leaf = 0;
  }
  return (int64_t)(iti ? plan_bytes<cplx>(&t, with_ws) : plan_bytes<double>(&t, with_ws));
}

// Peak device bytes of a recomputing handle with subtrees of depth d: the
// kept merges and subtree roots, the input copies, and one subtree built.
int64_t recompute_peak(int dim, int L, int p, int q, bool iti, int d, int64_t copies) {
  return uniform_plan(dim, L - d, p, q, iti, d, true) + uniform_plan(dim, d, p, q, iti, 0, true) + copies;
}

hps_tree subtree_of(const hps_handle* C, int64_t s, int d) {
  const int dim = C->dim, Ls = C->L - d;
  int64_t ix[3] = {0, 0, 0};
  for (int l = 0; l < Ls; ++l) {
    const int64_t c = (s >> (dim * (Ls - 1 - l))) & ((1 << dim) - 1);
    for (int a = 0; a < dim; ++a) ix[a] = 2 * ix[a] + ((c >> a) & 1);
  }
  hps_tree t{};
  t.dim = dim;
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      const double side = (C->hi[a] - C->lo[a]) / (double)((int64_t)1 << Ls);
      t.lo[a] = C->lo[a] + (double)ix[a] * side;
      t.hi[a] = t.lo[a] + side;
    } else {
      t.lo[a] = t.hi[a] = 0.0;
    }
  }
  t.uniform_depth = d;
  t.n_leaves = (int64_t)1 << (dim * d);
  t.morton = nullptr;
  t.level = nullptr;
  return t;
}

// Build subtree s (depth d) with the stored coefficients and source `f`
// (a full-tree array, or null); root_map asks for the root's T and h.
template <typename T>
hps_status build_subtree(hps_handle* C, int64_t s, const T* f, bool root_map, cudaStream_t st, hps_handle** out) {
  const int d = C->sub_depth;
  const int64_t lps = (int64_t)1 << (C->dim * d);
  const int64_t off = s * lps * C->npts;
  hps_tree t = subtree_of(C, s, d);
  hps_coeffs cf{};
  cf.kind = C->kind;
  cf.dtype = C->iti ? HPS_C128 : HPS_F64;
  cf.eta = C->eta;
  cf.a = C->rc_coef[0] ? C->rc_coef[0] + off : nullptr;
  for (int a = 0; a < 3; ++a) cf.b[a] = C->rc_coef[1 + a] ? C->rc_coef[1 + a] + off : nullptr;
  cf.c = C->rc_coef[4] ? C->rc_coef[4] + off : nullptr;
  hps_options o{};
  o.version = 1;
  o.want_root_map = root_map ? 1 : 0;
  o.iti_leaf = C->opts.iti_leaf;
  o.fp64_gemm = C->opts.fp64_gemm;
  return hps_build(&t, C->p, C->q, &cf, f ? (const void*)(f + off) : nullptr, &o, st, out);
}

template <typename T>
hps_status recompute_build(hps_handle* C, const hps_coeffs* cf, const void* f_in, int d, cudaStream_t st) {
  const int dim = C->dim;
  const int64_t n = C->nl * C->npts;
  C->recompute = true;
  C->sub_depth = d;
  // device copies of the inputs: the caller may release theirs after the build
  const double* src[5] = {cf->a, cf->b[0], cf->b[1], cf->b[2], cf->c};
  for (int i = 0; i < 5; ++i) {
    if (!src[i] || (i >= 1 && i <= 3 && i - 1 >= dim)) continue;
    double* dcp = (double*)dalloc(C, (size_t)n * sizeof(double));
    if (!dcp) return HPS_ERR_OOM;
    HPS_CUDA(cudaMemcpyAsync(dcp, src[i], (size_t)n * sizeof(double), cudaMemcpyDefault, st));
    C->rc_coef[i] = dcp;
  }
  if (f_in) {
    C->rc_f = dalloc(C, (size_t)n * sizeof(T));
    if (!C->rc_f) return HPS_ERR_OOM;
    HPS_CUDA(cudaMemcpyAsync(C->rc_f, f_in, (size_t)n * sizeof(T), cudaMemcpyDefault, st));
  }
  // the handle above the subtree roots
  hps_handle* Tp = new (std::nothrow) hps_handle();
  if (!Tp) return HPS_ERR_OOM;
  C->top = Tp;
  Tp->dim = dim; Tp->kind = C->kind; Tp->p = C->p; Tp->q = C->q; Tp->iti = C->iti;
  Tp->L = C->L - d;
  Tp->nl = (int64_t)1 << (dim * Tp->L);
  Tp->npts = C->npts;
  Tp->nroot = C->nroot;
  for (int a = 0; a < 3; ++a) { Tp->lo[a] = C->lo[a]; Tp->hi[a] = C->hi[a]; }
  Tp->hlen = C->hlen;
  Tp->eta = C->eta;
  Tp->opts = C->opts;
  Tp->num_sms = C->num_sms;
  Tp->device = C->device;
  Tp->last = st;
  Tp->ext_depth = d;
  if (cudaEventCreateWithFlags(&Tp->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return HPS_ERR_CUDA;
  }
  const int side = 1 << d;
  const int nbs = dim == 2 ? 4 * C->q * side : 6 * C->q * C->q * side * side;
  Tp->leafTH = dalloc(Tp, (size_t)Tp->nl * nbs * (nbs + 1) * sizeof(T));
  if (!Tp->leafTH) return HPS_ERR_OOM;
  // each subtree: leaf stage and merges to its root, keep the root's [T | h]
  for (int64_t s = 0; s < Tp->nl; ++s) {
    hps_handle* Hs = nullptr;
    HPS_TRY(build_subtree<T>(C, s, (const T*)C->rc_f, true, st, &Hs));
    const LevelDev& R = Hs->lev[d - 1];
    const bool ok = R.n_ext == nbs && R.nmerge == 1 && R.TP;
    cudaError_t e = ok ? cudaMemcpyAsync((T*)Tp->leafTH + s * (int64_t)nbs * (nbs + 1), R.TP,
                                         (size_t)nbs * (nbs + 1) * sizeof(T), cudaMemcpyDeviceToDevice, st)
                       : cudaSuccess;
    handle_end(Hs, st);
    hps_free(Hs);
    if (!ok) return HPS_ERR_INVALID;
    HPS_CUDA(e);
  }
  // the merges above the roots
  Tp->tcw.st = st;
  Tp->tcw.err_slot = &Tp->dev_err;
  Tp->tcw.enabled = C->opts.fp64_gemm == 0;
  hps_status s;
  {
    hps::TcScope tc_scope(&Tp->tcw);
    s = build_impl<T>(Tp, cf, nullptr, st);
  }
  if (Tp->tcw.p) {
    cudaStreamSynchronize(st);
    hps::tc_release(&Tp->tcw);
  }
  handle_end(Tp, st);
  if (s == HPS_ERR_SINGULAR) C->err_node = -1;
  return s;
}

template <typename T>
hps_status recompute_solve(hps_handle* C, int nrhs, const void* g_in, const void* f_in, void* u_out,
                           cudaStream_t st) {
  hps_handle* Tp = C->top;
  const int d = C->sub_depth;
  const int64_t lps = (int64_t)1 << (C->dim * d);
  const int64_t nsub = Tp->nl, npts = C->npts, nl = C->nl;
  const int nbs = Tp->nb;
  const size_t es = sizeof(T);
  // stage host buffers in the composite handle's own workspace
  const size_t gbytes = (size_t)C->nroot * nrhs * es, ubytes = (size_t)nl * npts * nrhs * es;
  if (C->ws_nrhs < nrhs) {
    for (void* pp : C->ws_allocs) dev_free(pp, st);
    C->ws_allocs.clear();
    C->ws_g = dalloc(C, gbytes, &C->ws_allocs);
    C->ws_f = dalloc(C, ubytes, &C->ws_allocs);
    C->ws_u = dalloc(C, ubytes, &C->ws_allocs);
    C->rc_u = dalloc(C, (size_t)lps * npts * nrhs * es, &C->ws_allocs);
    if (!C->ws_g || !C->ws_f || !C->ws_u || !C->rc_u) return HPS_ERR_OOM;
    C->ws_nrhs = nrhs;
  }
  const T* g = (const T*)g_in;
  if (!is_device_ptr(g_in)) {
    HPS_CUDA(cudaMemcpyAsync(C->ws_g, g_in, gbytes, cudaMemcpyHostToDevice, st));
    g = (const T*)C->ws_g;
  }
  const T* f = (const T*)f_in;
  if (f_in && !is_device_ptr(f_in)) {
    HPS_CUDA(cudaMemcpyAsync(C->ws_f, f_in, ubytes, cudaMemcpyHostToDevice, st));
    f = (const T*)C->ws_f;
  }
  const bool host_u = !is_device_ptr(u_out);
  T* u = host_u ? (T*)C->ws_u : (T*)u_out;
  handle_begin(Tp, st);
  HPS_TRY(ensure_ws<T>(Tp, nrhs));
  // new sources: each subtree rebuilt with the column's source gives its root's h
  if (f) {
    for (int64_t s = 0; s < nsub; ++s)
      for (int c = 0; c < nrhs; ++c) {
        hps_handle* Hs = nullptr;
        HPS_TRY(build_subtree<T>(C, s, f + (int64_t)c * nl * npts, true, st, &Hs));
        const LevelDev& R = Hs->lev[d - 1];
        cudaError_t e = cudaMemcpyAsync((T*)Tp->ws_hleaf + (s * nrhs + c) * (int64_t)nbs,
                                        (const T*)R.TP + (int64_t)nbs * nbs, (size_t)nbs * es,
                                        cudaMemcpyDeviceToDevice, st);
        handle_end(Hs, st);
        hps_free(Hs);
        HPS_CUDA(e);
      }
  }
  // upward pass above the roots (new sources), downward pass to the roots
  Tp->ext_newf = f != nullptr;
  hps_status rs = solve_impl<T>(Tp, nrhs, g, nullptr, Tp->ws_gleaf, st);
  Tp->ext_newf = false;
  handle_end(Tp, st);
  HPS_TRY(rs);
  // each subtree again: its downward pass and leaf output
  for (int64_t s = 0; s < nsub; ++s) {
    const T* gs = (const T*)Tp->ws_gleaf + s * (int64_t)nbs * nrhs;  // [nrhs][nbs]
    if (!f) {
      hps_handle* Hs = nullptr;
      HPS_TRY(build_subtree<T>(C, s, (const T*)C->rc_f, false, st, &Hs));
      hps_status ss = hps_solve_batched(Hs, nrhs, gs, nullptr, C->rc_u, st);
      cudaError_t e = cudaSuccess;
      if (ss == HPS_OK)
        e = cudaMemcpy2DAsync(u + s * lps * npts, (size_t)nl * npts * es, C->rc_u, (size_t)lps * npts * es,
                              (size_t)lps * npts * es, nrhs, cudaMemcpyDeviceToDevice, st);
      handle_end(Hs, st);
      hps_free(Hs);
      HPS_TRY(ss);
      HPS_CUDA(e);
    } else {
      for (int c = 0; c < nrhs; ++c) {
        hps_handle* Hs = nullptr;
        HPS_TRY(build_subtree<T>(C, s, f + (int64_t)c * nl * npts, false, st, &Hs));
        hps_status ss = hps_solve(Hs, gs + (int64_t)c * nbs, nullptr, u + (int64_t)c * nl * npts + s * lps * npts, st);
        hps_free(Hs);
        HPS_TRY(ss);
      }
    }
  }
  if (host_u) {
    HPS_CUDA(cudaMemcpyAsync(u_out, u, ubytes, cudaMemcpyDeviceToHost, st));
    HPS_CUDA(cudaStreamSynchronize(st));
  }
  return HPS_OK;
}

}  // namespace

thread_local int64_t g_last_err_node = -1;

void drop_graphs(hps_handle* h) {
  for (auto& e : h->graphs)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  h->graphs.clear();
}

// Wait for the handle's own work (not the whole device: other streams keep
// running), then give its memory back to the pool.
void free_handle(hps_handle* h) {
  if (!h) return;
  if (h->done && h->done_recorded) cudaEventSynchronize(h->done);
  if (h->top) free_handle(h->top);
  drop_graphs(h);
  for (void* p : h->ws_allocs) dev_free_idle(p);
  for (void* p : h->allocs) dev_free_idle(p);
  if (h->trsv_err_host) cudaFreeHost(h->trsv_err_host);
  if (h->done) cudaEventDestroy(h->done);
  cudaGetLastError();
  delete h;
}

// Order stream st after the handle's earlier work, and mark the end of the
// work a call enqueues.  Skipped while the stream is being captured into a
// graph by the caller (an event recorded outside a capture cannot be waited
// on inside it; the caller's graph orders the work itself).
static bool capturing_stream(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return cs != cudaStreamCaptureStatusNone;
}

void handle_begin(hps_handle* h, cudaStream_t st) {
  if (h->done && h->done_recorded && !capturing_stream(st)) {
    if (cudaStreamWaitEvent(st, h->done, 0) != cudaSuccess) cudaGetLastError();
  }
  h->last = st;
}

void handle_end(hps_handle* h, cudaStream_t st) {
  if (h->done && !capturing_stream(st)) {
    if (cudaEventRecord(h->done, st) == cudaSuccess) h->done_recorded = true;
    else cudaGetLastError();
  }
}

// Solve through a captured CUDA graph: the first call with a key runs
// eagerly (allocating the workspace), the second captures the enqueued work
// and every later call replays it.  The flag-ordered triangular solves are
// not captured (their epochs are host state); the blocked solves are.
hps_status graph_solve(hps_handle* h, int nrhs, const void* g, const void* f, void* u, cudaStream_t st) {
  auto eager = [&]() {
    return h->iti ? solve_impl<cplx>(h, nrhs, g, f, u, st) : solve_impl<double>(h, nrhs, g, f, u, st);
  };
  if (h->trsv_err_host && *(volatile int*)h->trsv_err_host) return HPS_ERR_TIMEOUT;
  for (size_t i = 0; i < h->graphs.size(); ++i) {
    auto& e = h->graphs[i];
    if (e.nrhs != nrhs || e.g != g || e.f != f || e.u != u) continue;
    if (e.exec) {
      HPS_CUDA(cudaGraphLaunch(e.exec, st));
      return HPS_OK;
    }
    // second call: capture
    cudaGraph_t graph = nullptr;
    HPS_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    hps_status s = eager();
    h->capturing = false;
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (s != HPS_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return s != HPS_OK ? s : HPS_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      return HPS_ERR_CUDA;
    }
    e.exec = exec;
    HPS_CUDA(cudaGraphLaunch(e.exec, st));
    return HPS_OK;
  }
  // first call with this key: run eagerly, remember the key
  hps_status s = eager();
  if (s != HPS_OK) return s;
  if (h->graphs.size() >= 8) {
    if (h->graphs.front().exec) cudaGraphExecDestroy(h->graphs.front().exec);
    h->graphs.erase(h->graphs.begin());
  }
  hps_handle::GraphEntry e;
  e.nrhs = nrhs;
  e.g = g;
  e.f = f;
  e.u = u;
  e.warm = true;
  h->graphs.push_back(e);
  return HPS_OK;
}

}  // namespace

hps_status hps::ensure_solve_ws(hps_handle* h, int nrhs) {
  return h->iti ? ensure_ws<cplx>(h, nrhs) : ensure_ws<double>(h, nrhs);
}

namespace hps {
std::atomic<int64_t>& alloc_fail_countdown() {
  static std::atomic<int64_t> c{0};
  return c;
}
std::atomic<int64_t>& alloc_counter() {
  static std::atomic<int64_t> c{0};
  return c;
}
}  // namespace hps

extern "C" {

const char* hps_error_string(hps_status s) {
  switch (s) {
    case HPS_OK: return "HPS_OK: success";
    case HPS_ERR_INVALID: return "HPS_ERR_INVALID: invalid argument";
    case HPS_ERR_OOM: return "HPS_ERR_OOM: not enough device memory";
    case HPS_ERR_SINGULAR: return "HPS_ERR_SINGULAR: zero pivot in a leaf or merge factorisation";
    case HPS_ERR_CUDA: return "HPS_ERR_CUDA: a CUDA runtime call failed";
    case HPS_ERR_TIMEOUT: return "HPS_ERR_TIMEOUT: a bounded device-side wait gave up";
    case HPS_PENDING: return "HPS_PENDING: the request has not finished";
  }
  return "unknown hps_status";
}

hps_status hps_refine(const double lo[3], const double hi[3], int p, double eps, int min_depth, int max_depth,
                      int n_fn, const hps_eval_fn* fns, void* const* ctxs, int64_t capacity, int64_t* n_leaves,
                      uint64_t* morton, int8_t* level, struct CUstream_st* stream) {
  try {
    return adaptive_refine(lo, hi, p, eps, min_depth, max_depth, n_fn, fns, ctxs, capacity, n_leaves, morton,
                           level, (cudaStream_t)stream);
  } catch (...) {
    return HPS_ERR_INVALID;
  }
}

hps_status hps_sizes(const hps_tree* tree, int p, int q, int64_t* n_leaves, int64_t* ppl, int64_t* nroot) {
  if (tree && tree->uniform_depth == -1) {
    ATree at;
    hps_status s = adaptive_tree_from_abi(tree, p, q, &at);
    if (s != HPS_OK) return s;
    if (n_leaves) *n_leaves = tree->n_leaves;
    if (ppl) *ppl = (int64_t)p * p * p;
    if (nroot) *nroot = at.nodes[0].n_bdry;
    return HPS_OK;
  }
  hps_status s = check_tree(tree, p, q);
  if (s != HPS_OK) return s;
  const int L = tree->uniform_depth, d = tree->dim;
  if (n_leaves) *n_leaves = (int64_t)1 << (d * L);
  if (ppl) *ppl = d == 2 ? (int64_t)p * p : (int64_t)p * p * p;
  if (nroot) *nroot = nroot_of(d, q, L);
  return HPS_OK;
}

hps_status hps_nodes(const hps_tree* tree, int p, int q, double* leaf_xyz, double* bdry_xyz) {
  if (tree && tree->uniform_depth == -1) {
    ATree at;
    hps_status s = adaptive_tree_from_abi(tree, p, q, &at);
    if (s != HPS_OK) return s;
    Spectral1D sp = make_spectral(p, q);
    if (leaf_xyz) atree_leaf_coords(at, sp, leaf_xyz);
    if (bdry_xyz) atree_root_coords(at, sp, bdry_xyz);
    return HPS_OK;
  }
  hps_status s = check_tree(tree, p, q);
  if (s != HPS_OK) return s;
  try {
    Spectral1D sp = make_spectral(p, q);
    if (leaf_xyz) leaf_node_coords(tree->dim, tree->lo, tree->hi, tree->uniform_depth, sp, leaf_xyz);
    if (bdry_xyz) root_boundary_coords(tree->dim, tree->lo, tree->hi, tree->uniform_depth, sp, bdry_xyz);
  } catch (...) {
    return HPS_ERR_INVALID;
  }
  return HPS_OK;
}

hps_status hps_build(const hps_tree* tree, int p, int q, const hps_coeffs* coeffs, const void* f,
                     const hps_options* opts, struct CUstream_st* stream, hps_handle** out) {
  if (!out) return HPS_ERR_INVALID;
  *out = nullptr;
  const bool adaptive = tree && tree->uniform_depth == -1;
  hps_status s = HPS_OK;
  int64_t a_nroot = 0;
  if (adaptive) {
    int64_t nl = 0, ppl = 0;
    s = hps_sizes(tree, p, q, &nl, &ppl, &a_nroot);
    if (s != HPS_OK) return s;
    if (!coeffs || coeffs->kind != HPS_DTN) return HPS_ERR_INVALID;
  } else {
    s = check_tree(tree, p, q);
  }
  if (s != HPS_OK) return s;
  if (!coeffs) return HPS_ERR_INVALID;
  if (coeffs->kind != HPS_DTN && coeffs->kind != HPS_ITI) return HPS_ERR_INVALID;
  if (coeffs->kind == HPS_DTN && coeffs->dtype != HPS_F64) return HPS_ERR_INVALID;
  if (coeffs->kind == HPS_ITI && (coeffs->dtype != HPS_C128 || tree->dim != 2 || !(coeffs->eta > 0)))
    return HPS_ERR_INVALID;
  if (opts && opts->version != 1) return HPS_ERR_INVALID;
  hps_handle* h = new (std::nothrow) hps_handle();
  if (!h) return HPS_ERR_OOM;
  h->dim = tree->dim; h->kind = coeffs->kind; h->p = p; h->q = q; h->L = tree->uniform_depth;
  h->iti = coeffs->kind == HPS_ITI;
  h->nl = (int64_t)1 << (h->dim * h->L);
  h->npts = h->dim == 2 ? (int64_t)p * p : (int64_t)p * p * p;
  h->nroot = nroot_of(h->dim, q, h->L);
  for (int a = 0; a < 3; ++a) { h->lo[a] = tree->lo[a]; h->hi[a] = tree->hi[a]; }
  h->hlen = (tree->hi[0] - tree->lo[0]) / (double)((int64_t)1 << h->L);
  h->eta = coeffs->eta;
  if (adaptive) {
    h->adaptive = true;
    h->L = 0;
    h->nl = tree->n_leaves;
    h->npts = (int64_t)p * p * p;
    h->nroot = a_nroot;
    h->hlen = 0.0;
  }
  if (opts) h->opts = *opts;
  else { h->opts.version = 1; h->opts.want_root_map = 0; h->opts.profile = 0; }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return HPS_ERR_CUDA;
  }
  h->device = dev;
  if (cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return HPS_ERR_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  h->last = st;
  h->tcw.st = st;
  h->tcw.err_slot = &h->dev_err;
  h->tcw.enabled = h->opts.fp64_gemm == 0;
  // subtree recomputation when the planned footprint exceeds the budget
  int rc_depth = 0;
  if (!h->adaptive && h->opts.recompute_budget_mb > 0 && h->L >= 2) {
    const int64_t budget = (int64_t)h->opts.recompute_budget_mb << 20;
    if (uniform_plan(h->dim, h->L, p, q, h->iti, 0, true) > budget) {
      const int64_t n = h->nl * h->npts;
      const int64_t copies = (int64_t)(h->dim + 2) * n * 8 + (f ? n * (h->iti ? 16 : 8) : 0);
      for (int d = h->L - 1; d >= 1 && !rc_depth; --d)
        if (recompute_peak(h->dim, h->L, p, q, h->iti, d, copies) <= budget) rc_depth = d;
      if (!rc_depth) {
        handle_end(h, st);
        free_handle(h);
        return HPS_ERR_OOM;
      }
    }
  }
  try {
    hps::TcScope tc_scope(&h->tcw);
    if (h->adaptive) s = adaptive_build(h, tree, coeffs, f, st);
    else if (rc_depth)
      s = h->iti ? recompute_build<cplx>(h, coeffs, f, rc_depth, st) : recompute_build<double>(h, coeffs, f, rc_depth, st);
    else s = h->iti ? build_impl<cplx>(h, coeffs, f, st) : build_impl<double>(h, coeffs, f, st);
  } catch (...) {
    s = HPS_ERR_INVALID;
  }
  // the digit-slice workspace only lives through the build
  if (h->tcw.p) {
    cudaStreamSynchronize(st);
    hps::tc_release(&h->tcw);
  }
  // a failed build may leave work queued on st: free_handle waits for it
  if (s != HPS_OK) handle_end(h, st);
  if (s != HPS_OK && s != HPS_ERR_SINGULAR) {
    free_handle(h);
    return s;
  }
  if (s == HPS_ERR_SINGULAR) {
    // no half-built handle is returned; the node id stays readable through
    // hps_last_error_detail(NULL, &node) on this thread
    g_last_err_node = h->err_node;
    free_handle(h);
    return s;
  }
  g_last_err_node = -1;
  handle_end(h, st);
  *out = h;
  return HPS_OK;
}

hps_status hps_solve_batched(hps_handle* h, int nrhs, const void* g, const void* f, void* u,
                             struct CUstream_st* stream) {
  if (!h || !g || !u || nrhs < 1) return HPS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  handle_begin(h, st);
  hps_status s;
  try {
    if (h->recompute)
      s = h->iti ? recompute_solve<cplx>(h, nrhs, g, f, u, st) : recompute_solve<double>(h, nrhs, g, f, u, st);
    else if (h->adaptive) s = adaptive_solve(h, nrhs, g, f, u, st);
    else if (h->opts.graph_solve && !h->opts.profile && st && is_device_ptr(g) && is_device_ptr(u) &&
             (!f || is_device_ptr(f)))
      s = graph_solve(h, nrhs, g, f, u, st);
    else s = h->iti ? solve_impl<cplx>(h, nrhs, g, f, u, st) : solve_impl<double>(h, nrhs, g, f, u, st);
  } catch (...) {
    h->capturing = false;
    s = HPS_ERR_INVALID;
  }
  handle_end(h, st);
  return s;
}

hps_status hps_solve_multi(int n, hps_handle* const* hs, const int* nrhs, const void* const* g, void* const* u,
                           struct CUstream_st* stream) {
  if (n < 1 || n > 1024 || !hs || !nrhs || !g || !u) return HPS_ERR_INVALID;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HPS_ERR_CUDA;
  }
  std::vector<int> real_idx, cplx_idx;
  for (int i = 0; i < n; ++i) {
    hps_handle* h = hs[i];
    if (!h || h->adaptive || h->recompute || nrhs[i] < 1 || !g[i] || !u[i] || h->device != dev)
      return HPS_ERR_INVALID;
    for (int j = 0; j < i; ++j)
      if (hs[j] == h) return HPS_ERR_INVALID;
    if (!is_device_ptr(g[i]) || !is_device_ptr(u[i])) return HPS_ERR_INVALID;
    (h->iti ? cplx_idx : real_idx).push_back(i);
  }
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < n; ++i) handle_begin(hs[i], st);
  hps_status s = HPS_OK;
  try {
    if (!real_idx.empty()) s = solve_multi_impl<double>(real_idx, hs, nrhs, g, u, st);
    if (s == HPS_OK && !cplx_idx.empty()) s = solve_multi_impl<cplx>(cplx_idx, hs, nrhs, g, u, st);
  } catch (...) {
    s = HPS_ERR_INVALID;
  }
  for (int i = 0; i < n; ++i) handle_end(hs[i], st);
  return s;
}

hps_status hps_solve(hps_handle* h, const void* g, const void* f, void* u, struct CUstream_st* stream) {
  return hps_solve_batched(h, 1, g, f, u, stream);
}

hps_status hps_solve_adjoint(hps_handle* h, int nrhs, const void* ubar, void* gbar, void* fbar,
                             struct CUstream_st* stream) {
  if (!h || !ubar || nrhs < 1 || h->adaptive || h->recompute) return HPS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  handle_begin(h, st);
  hps_status s;
  try {
    s = adjoint_solve(h, nrhs, ubar, gbar, fbar, st);
  } catch (...) {
    s = HPS_ERR_INVALID;
  }
  handle_end(h, st);
  return s;
}

hps_status hps_debug_wait_timeout(int which, int satisfied, int64_t limit_polls, struct CUstream_st* stream) {
  if (which < 0 || which > 2 || limit_polls < 1 || limit_polls > ((int64_t)1 << 24)) return HPS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* d = nullptr;  // words[0..2] waited on, words[3] the status word
  HPS_CUDA(cudaMalloc(&d, 4 * sizeof(unsigned)));
  cudaError_t e = cudaMemsetAsync(d, 0, 4 * sizeof(unsigned), st);
  if (e == cudaSuccess)
    e = which == 2 ? hps::debug_mbar_wait(satisfied ? 1 : 0, (long)limit_polls, d + 3, st)
                   : hps::debug_wait(which, satisfied ? 1 : 0, d, (unsigned long long)limit_polls, d + 3, st);
  unsigned herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d + 3, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HPS_ERR_CUDA;
  }
  return (herr & hps::DEV_ERR_TIMEOUT) ? HPS_ERR_TIMEOUT : HPS_OK;
}

hps_status hps_tune_set(int param, int value) {
  if (param < 0 || param >= hps::TUNE_COUNT || value < 0 || value > (1 << 20)) return HPS_ERR_INVALID;
  hps::lu_tune(param) = value;
  return HPS_OK;
}

hps_status hps_tune_get(int param, int* value) {
  if (param < 0 || param >= hps::TUNE_COUNT || !value) return HPS_ERR_INVALID;
  *value = hps::lu_tune(param);
  return HPS_OK;
}

void hps_debug_fail_alloc(int64_t n) { hps::alloc_fail_countdown().store(n > 0 ? n : 0); }

int64_t hps_debug_alloc_count(void) { return hps::alloc_counter().load(); }

hps_status hps_gemm(int dtype, int mode, int m, int n, int k, int batch, double alpha, const void* A, int lda,
                    int64_t strideA, const void* B, int ldb, int64_t strideB, double beta, void* C, int ldc,
                    int64_t strideC, struct CUstream_st* stream) {
  if ((dtype != HPS_F64 && dtype != HPS_C128) || (mode != 0 && mode != 1)) return HPS_ERR_INVALID;
  if (m < 0 || n < 0 || k < 0 || batch < 0 || !A || !B || !C) return HPS_ERR_INVALID;
  if (lda < std::max(m, 1) || ldb < std::max(k, 1) || ldc < std::max(m, 1)) return HPS_ERR_INVALID;
  if (m == 0 || n == 0 || batch == 0) return HPS_OK;
  if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C)) return HPS_ERR_INVALID;
  // an empty inner dimension leaves C = beta C; only beta 0 or 1 is supported there
  if (k == 0 && beta != 0.0 && beta != 1.0) return HPS_ERR_INVALID;
  if (k == 0 && beta == 1.0) return HPS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* derr = nullptr;
  HPS_CUDA(cudaMalloc(&derr, sizeof(unsigned)));
  hps::TcWorkspace w;
  w.err_slot = &derr;
  w.enabled = mode == 0;
  w.force = true;
  cudaError_t e = cudaMemsetAsync(derr, 0, sizeof(unsigned), st);
  {
    hps::TcScope scope(&w);
    auto run = [&](auto* tag) -> cudaError_t {
      using T = std::remove_pointer_t<decltype(tag)>;
      hps::GemmArgs<T> g;
      g.M = m; g.N = n; g.K = k; g.batch = batch;
      g.A = hps::bop<T>((T*)A, strideA, lda);
      g.B = hps::bop<T>((T*)B, strideB, ldb);
      g.C = hps::bop<T>((T*)C, strideC, ldc);
      g.alpha = T(alpha);
      g.beta = T(beta);
      if (k == 0) return hps::fill<T>(g.C, m, n, batch, T(0.0), T(0.0), st, nullptr);
      return hps::gemm<T>(g, st, nullptr);
    };
    if (e == cudaSuccess) e = dtype == HPS_F64 ? run((double*)nullptr) : run((hps::cplx*)nullptr);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  unsigned herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost);
  hps::tc_release(&w);
  cudaFree(derr);
  if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return HPS_ERR_OOM; }
  if (e != cudaSuccess) { cudaGetLastError(); return HPS_ERR_CUDA; }
  return (herr & hps::DEV_ERR_TIMEOUT) ? HPS_ERR_TIMEOUT : HPS_OK;
}

hps_status hps_getrf(int dtype, int mode, int n, int batch, void* A, int lda, int64_t strideA, int* ipiv,
                     int* info, struct CUstream_st* stream) {
  if ((dtype != HPS_F64 && dtype != HPS_C128) || (mode != 0 && mode != 1)) return HPS_ERR_INVALID;
  if (n < 0 || batch < 0 || !A || !ipiv || !info || lda < std::max(n, 1)) return HPS_ERR_INVALID;
  if (batch > 1 && strideA < (int64_t)lda * n) return HPS_ERR_INVALID;
  if (n == 0 || batch == 0) return HPS_OK;
  if (batch > (1 << 30) / std::max(n, 1)) return HPS_ERR_INVALID;
  if (!is_device_ptr(A) || !is_device_ptr(ipiv) || !is_device_ptr(info)) return HPS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  HPS_CUDA(cudaGetDevice(&dev));
  HPS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const bool cp = dtype == HPS_C128;
  const int G = cp ? hps::lu_group_size<hps::cplx>(n, batch, sms) : hps::lu_group_size<double>(n, batch, sms);
  hps::LuWork luw;
  luw.pub_bytes = cp ? hps::lu_pub_bytes<hps::cplx>(n, batch, G) : hps::lu_pub_bytes<double>(n, batch, G);
  unsigned* derr = nullptr;
  int* perm = nullptr;
  cudaError_t e = cudaMalloc(&derr, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&perm, sizeof(int) * (size_t)batch * n);
  if (e == cudaSuccess) e = cudaMalloc(&luw.bars, sizeof(unsigned) * 2 * (size_t)batch);
  if (e == cudaSuccess && luw.pub_bytes) e = cudaMalloc(&luw.pub, luw.pub_bytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(derr, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(luw.bars, 0, sizeof(unsigned) * 2 * (size_t)batch, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(info, 0, sizeof(int) * (size_t)batch, st);
  hps::TcWorkspace w;
  w.err_slot = &derr;
  w.enabled = mode == 0;
  if (e == cudaSuccess) {
    hps::TcScope scope(&w);
    if (cp) e = hps::getrf<hps::cplx>(hps::bop<hps::cplx>((hps::cplx*)A, strideA, lda), n, batch, ipiv, perm, info, derr, G, luw, st,
                                 nullptr);
    else e = hps::getrf<double>(hps::bop<double>((double*)A, strideA, lda), n, batch, ipiv, perm, info, derr, G, luw,
                                st, nullptr);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  unsigned herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(unsigned), cudaMemcpyDeviceToHost);
  hps::tc_release(&w);
  if (e != cudaSuccess) cudaStreamSynchronize(st);
  cudaFree(luw.pub);
  cudaFree(luw.bars);
  cudaFree(perm);
  cudaFree(derr);
  if (e == cudaErrorMemoryAllocation) { cudaGetLastError(); return HPS_ERR_OOM; }
  if (e != cudaSuccess) { cudaGetLastError(); return HPS_ERR_CUDA; }
  return (herr & hps::DEV_ERR_TIMEOUT) ? HPS_ERR_TIMEOUT : HPS_OK;
}

hps_status hps_coeff_gradient(hps_handle* h, int nrhs, const void* u, const void* fbar, double* ga, double* gb,
                              double* gc, struct CUstream_st* stream) {
  if (!h || !u || !fbar || nrhs < 1 || h->adaptive || h->recompute) return HPS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  handle_begin(h, st);
  const hps_status s = coeff_gradient(h, nrhs, u, fbar, ga, gb, gc, st);
  handle_end(h, st);
  return s;
}

void hps_free(hps_handle* h) { free_handle(h); }

hps_status hps_last_error_detail(hps_handle* h, int64_t* node) {
  if (!node) return HPS_ERR_INVALID;
  *node = h ? h->err_node : g_last_err_node;
  return HPS_OK;
}

int64_t hps_device_bytes(const hps_handle* h) { return h ? h->bytes + (h->top ? h->top->bytes : 0) : 0; }

hps_status hps_plan_bytes(const hps_tree* tree, int p, int q, int kind, int64_t* bytes) {
  if (!bytes) return HPS_ERR_INVALID;
  *bytes = 0;
  hps_status s = check_tree(tree, p, q);
  if (s != HPS_OK) return s;
  if (kind != HPS_DTN && kind != HPS_ITI) return HPS_ERR_INVALID;
  if (kind == HPS_ITI && tree->dim != 2) return HPS_ERR_INVALID;
  hps_handle h;
  h.dim = tree->dim; h.p = p; h.q = q; h.L = tree->uniform_depth; h.iti = kind == HPS_ITI;
  h.nl = (int64_t)1 << (h.dim * h.L);
  h.npts = h.dim == 2 ? (int64_t)p * p : (int64_t)p * p * p;
  const int64_t ni = h.dim == 2 ? (int64_t)(p - 2) * (p - 2) : (int64_t)(p - 2) * (p - 2) * (p - 2);
  h.nb = h.dim == 2 ? 4 * q : 6 * q * q;
  h.nlu_leaf = (int)(h.iti ? h.npts : ni);
  h.xrows_leaf = h.nlu_leaf;
  const size_t b = h.iti ? plan_bytes<cplx>(&h, true) : plan_bytes<double>(&h, true);
  *bytes = (int64_t)b;
  return HPS_OK;
}

int64_t hps_last_launch_count(const hps_handle* h) { return h ? h->prof.launches : 0; }

hps_status hps_kernel_stats(hps_handle* h, int cls, hps_kernel_stat* out) {
  if (!h || !out || cls < 0 || cls >= HPS_KCLASS_COUNT) return HPS_ERR_INVALID;
  if (h->prof.on && cudaStreamSynchronize(h->last) != cudaSuccess) return HPS_ERR_CUDA;
  out->launches = h->prof.n[cls];
  out->flops = h->prof.flops[cls];
  out->ms = h->prof.on ? h->prof.ms(cls) : -1.0;
  out->exec_flops = h->prof.exec[cls];
  return HPS_OK;
}

hps_status hps_set_profiling(hps_handle* h, int on) {
  if (!h) return HPS_ERR_INVALID;
  h->opts.profile = on ? 1 : 0;
  return HPS_OK;
}

hps_status hps_trace_count(hps_handle* h, int64_t* count) {
  if (!h || !count) return HPS_ERR_INVALID;
  if (h->prof.on && cudaStreamSynchronize(h->last) != cudaSuccess) return HPS_ERR_CUDA;
  *count = (int64_t)h->prof.trace.size();
  return HPS_OK;
}

hps_status hps_trace_get(hps_handle* h, int64_t i, hps_trace_rec* out) {
  if (!h || !out || i < 0 || i >= (int64_t)h->prof.trace.size()) return HPS_ERR_INVALID;
  const Prof::Rec& r = h->prof.trace[(size_t)i];
  out->kclass = r.cls;
  out->m = r.m;
  out->n = r.n;
  out->k = r.k;
  out->batch = r.batch;
  out->flops = r.flops;
  out->ms = h->prof.rec_ms(r);
  return HPS_OK;
}

}  // extern "C"

// ----------------------------------------------------------------------------
// Allocation-free solve.  Some callers cannot let a library allocate device
// memory: code that runs inside a memory budget owned by another allocator
// (a framework's caching pool, a serving process that reserves all memory up
// front) or code that must not call cudaMalloc / cudaFree at that point
// because they synchronise the device.  hps_solve allocates its per-level
// vectors lazily in the handle; hps_solve_noalloc runs the same downward pass
// and leaf output with those vectors placed in one static device array
// instead, so the call itself allocates nothing.
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;  // 16 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kNoAllocMaxDevices = 64;
// Per-device address cache.  Two host threads making the first call on one
// device at the same time may both look the address up; they store the same
// value, and the atomics keep that free of data races.
std::atomic<void*> g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the static array on device `dev` (the current device).
// In host code the symbol names a host-side stand-in, so the address must
// come from cudaGetSymbolAddress, once per device, with that device current.
hps_status noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return HPS_ERR_INVALID;
  void* p = g_noalloc_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HPS_ERR_CUDA;
    }
    g_noalloc_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return HPS_OK;
}

// True when p is device (or managed) memory that the current device `dev`
// can use directly: allocated on dev, or managed.
bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

template <typename T>
hps_status solve_noalloc_impl(hps_handle* h, int dev, const T* g, T* u, cudaStream_t st) {
  // scratch layout: per level (from the root down) g_int then the children's g
  const size_t al = 256 / sizeof(T);
  auto up = [&](size_t n) { return (n + al - 1) / al * al; };
  size_t need = 0;
  for (int m = h->L - 1; m >= 0; --m) {
    const LevelDev& Lv = h->lev[m];
    need += up((size_t)Lv.nmerge * Lv.n_int) + up((size_t)Lv.nmerge * Lv.nch * Lv.nbc);
  }
  if (need * sizeof(T) > kNoAllocScratchBytes) return HPS_ERR_INVALID;
  void* base = nullptr;
  hps_status s = noalloc_scratch(dev, &base);
  if (s != HPS_OK) return s;
  T* cur = reinterpret_cast<T*>(base);
  const T* gpar = g;
  for (int m = h->L - 1; m >= 0; --m) {
    LevelDev& Lv = h->lev[m];
    T* gint = cur;
    cur += up((size_t)Lv.nmerge * Lv.n_int);
    T* gchild = cur;
    cur += up((size_t)Lv.nmerge * Lv.nch * Lv.nbc);
    HPS_CUDA(down_level<T>((const T*)Lv.X, nullptr, gpar, Lv.nmerge, Lv.nch, Lv.nbc, Lv.n_ext, Lv.n_int, 1,
                           Lv.ext, Lv.var, gint, gchild, st, nullptr));
    gpar = gchild;
  }
  HPS_CUDA(leaf_output<T>(h->lc, h->nl, 1, (const T*)h->leafX, nullptr, gpar, u, Kind<T>::iti, st, nullptr));
  return HPS_OK;
}

}  // namespace

extern "C" hps_status hps_solve_noalloc(hps_handle* h, const void* g, void* u, struct CUstream_st* stream) {
  if (!h || !g || !u || h->adaptive || h->recompute || (h->L > 0 && h->lev[h->L - 1].lazy))
    return HPS_ERR_INVALID;
  // the handle, g and u must all live on the current device: a kernel given
  // pointers of another device would fault
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HPS_ERR_CUDA;
  }
  if (dev != h->device || !on_device(g, dev) || !on_device(u, dev)) return HPS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  handle_begin(h, st);
  hps_status s;
  try {
    s = h->iti ? solve_noalloc_impl<cplx>(h, dev, (const cplx*)g, (cplx*)u, st)
               : solve_noalloc_impl<double>(h, dev, (const double*)g, (double*)u, st);
  } catch (...) {
    s = HPS_ERR_INVALID;
  }
  handle_end(h, st);
  return s;
}
