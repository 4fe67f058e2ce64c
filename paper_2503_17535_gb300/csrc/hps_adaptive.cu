// Adaptive 3D DtN build and solve (Section 4.2): the leaf stage with
// per-leaf sizes, then the nonuniform merges one merge node at a time, deepest
// level first: each child's [T | h] is projected onto the coarsened interfaces
// (4-to-1 panel projections), gathered into D, [C | h_int] and [A | h_ext],
// D is factored (a cooperative group of CTAs), X = D^{-1}[C | h_int] and
// [T | h] = [A | h_ext] - B X with one gathered product per child.  The
// downward pass interpolates interface data back onto fine panels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "handle.h"
#include "hps_adaptive.h"

namespace hps {

namespace {

template <typename V>
V* up_vec(hps_handle* h, const std::vector<V>& v, cudaStream_t st) {
  return upload(h, v, st);
}

const double* child_T(hps_handle* h, int child_node, int* n, int* ld) {
  const ANode& K = h->at.nodes[child_node];
  if (K.leaf >= 0) {
    *n = h->nb;
    *ld = h->nb;
    return (const double*)h->leafTH + (int64_t)K.leaf * h->nb * (h->nb + 1);
  }
  const AMergeDev& M = h->am[h->node_merge[child_node]];
  *n = M.n_ext;
  *ld = M.n_ext;
  return (const double*)M.TP;
}

}  // namespace

hps_status adaptive_tree_from_abi(const hps_tree* t, int p, int q, ATree* out) {
  if (!t || t->dim != 3 || t->uniform_depth != -1 || !t->morton || !t->level || t->n_leaves < 1)
    return HPS_ERR_INVALID;
  if (p < 4 || p > 24 || q != p - 2) return HPS_ERR_INVALID;
  const double side = t->hi[0] - t->lo[0];
  if (!(side > 0)) return HPS_ERR_INVALID;
  for (int a = 1; a < 3; ++a)
    if (!(std::fabs((t->hi[a] - t->lo[a]) - side) <= 1e-12 * side)) return HPS_ERR_INVALID;
  const char* why = nullptr;
  try {
    if (!build_atree(p, q, t->lo, t->hi, t->n_leaves, t->morton, t->level, out, &why)) return HPS_ERR_INVALID;
  } catch (...) {
    return HPS_ERR_INVALID;
  }
  return HPS_OK;
}

// C <- C - B X for every member of a group, per child position: X (n_int
// rows, N columns) and C (n_ext rows) of each member through the pointer
// arrays dXs / dCs; in the build, C = [T | h] (skipped for the root unless
// the root map is wanted); in the solve, C = h_ext.
static hps_status group_b_products(hps_handle* h, const AGroup& A, double** dXs, int N, double** dCs, bool build,
                                   cudaStream_t st, Prof* pf) {
  using T = double;
  const int nbat = (int)A.members.size();
  for (int c = 0; c < 8; ++c) {
    const AGroup::ChildBatch& cb = A.cb[c];
    if (cb.ok) {
      GemmArgs<T> g;
      g.M = cb.ne_c; g.N = N; g.K = cb.ni_c; g.batch = nbat;
      g.A = bopp<T>(cb.dTp, cb.np);
      g.arow.idx = cb.barow; g.arow.len = cb.ne_c; g.arow.period = nbat;
      g.acol.idx = cb.bacol; g.acol.len = cb.ni_c; g.acol.period = nbat;
      g.B = bopp<T>(dXs, A.n_int);
      g.brow.idx = cb.bbrow; g.brow.len = cb.ni_c; g.brow.period = nbat;
      g.C = bopp<T>(dCs, A.n_ext);
      g.crow.idx = cb.bcrow; g.crow.len = cb.ne_c; g.crow.period = nbat;
      g.alpha = -1.0; g.beta = 1.0;
      HPS_CUDA(gemm<T>(g, st, pf));
      continue;
    }
    for (int k2 = 0; k2 < nbat; ++k2) {
      const AMergeDev& M = h->am[(size_t)A.members[k2]];
      if (M.node == 0 && !(build && h->opts.want_root_map)) continue;
      const AChildDev& CD = M.ch[c];
      GemmArgs<T> g;
      g.M = CD.ne_c; g.N = N; g.K = CD.ni_c; g.batch = 1;
      g.A = bop<T>((T*)CD.Tp, 0, CD.pj.np);
      g.arow.idx = CD.barow; g.arow.len = CD.ne_c;
      g.acol.idx = CD.bacol; g.acol.len = CD.ni_c;
      g.B = bopp<T>(dXs, M.n_int);
      g.B.ptrs = dXs + k2;
      g.brow.idx = CD.bbrow; g.brow.len = CD.ni_c;
      g.C = bopp<T>(dCs + k2, M.n_ext);
      g.crow.idx = CD.bcrow; g.crow.len = CD.ne_c;
      g.alpha = -1.0; g.beta = 1.0;
      HPS_CUDA(gemm<T>(g, st, pf));
    }
  }
  return HPS_OK;
}

hps_status adaptive_build(hps_handle* h, const hps_tree* tree, const hps_coeffs* cf, const void* f_in,
                          cudaStream_t st) {
  using T = double;
  Prof* pf = &h->prof;
  pf->reset();
  pf->on = h->opts.profile != 0;
  hps_status rs = adaptive_tree_from_abi(tree, h->p, h->q, &h->at);
  if (rs != HPS_OK) return rs;
  ATree& at = h->at;
  const int p = h->p, q = h->q, q2 = q * q;
  h->spec = make_spectral(p, q);
  h->dref = make_dtn_leaf(h->spec, 3);
  h->nb = h->dref.nb;
  h->nlu_leaf = h->dref.ni;
  h->xrows_leaf = h->dref.ni;
  const int64_t nl = h->nl;
  const int nb = h->nb, ni = h->dref.ni;
  // ---- footprint check
  size_t need = (size_t)nl * ((size_t)ni * ni + (size_t)ni * (nb + 1) + (size_t)nb * (nb + 1)) * sizeof(T);
  size_t scratch_R = (size_t)nl * ni * (nb + 1), tmp = 0;
  int max_np = 0;
  {
    // the merges of one level keep their [C | h_int] side by side
    std::vector<size_t> per_level((size_t)at.max_level + 1, 0);
    for (const MergePlanA& pl : at.plans)
      per_level[(size_t)at.nodes[pl.node].level] += (size_t)pl.n_int * (pl.n_ext + 1);
    for (size_t v : per_level) scratch_R = std::max(scratch_R, v);
  }
  for (const MergePlanA& pl : at.plans) {
    need += ((size_t)pl.n_ext * (pl.n_ext + 1) + (size_t)pl.n_int * pl.n_int + (size_t)pl.n_int * (pl.n_ext + 1)) *
            sizeof(T);
    for (int c = 0; c < 8; ++c) {
      need += (size_t)pl.ch[c].np * (pl.ch[c].np + 1) * sizeof(T);
      tmp = std::max(tmp, (size_t)pl.ch[c].n * (pl.ch[c].np + 1));
      max_np = std::max(max_np, pl.ch[c].np);
    }
  }
  need += (scratch_R + tmp) * sizeof(T) + ((size_t)64 << 20);
  {
    size_t fr = 0, tot = 0;
    HPS_CUDA(cudaMemGetInfo(&fr, &tot));
    if (need > fr + dev_pool_idle_bytes()) return HPS_ERR_OOM;
  }
  h->max_np = max_np;
  // ---- constants
  h->dD = upload(h, h->spec.D, st);
  h->dDD = upload(h, h->spec.DD, st);
  std::vector<int> iidx(h->npts, -1);
  for (int i = 0; i < ni; ++i) iidx[h->dref.Ii[i]] = i;
  h->dIi = upload(h, h->dref.Ii, st);
  h->dprow = upload(h, h->dref.prow, st);
  h->dP = upload(h, h->dref.P, st);
  h->dQi = upload(h, h->dref.Qi, st);
  h->dQP = upload(h, h->dref.QP, st);
  h->diidx = upload(h, iidx, st);
  std::vector<double> sl(nl), C2F, F2C;
  for (int64_t n = 0; n < nl; ++n) sl[n] = 2.0 / (at.side / (double)((int64_t)1 << at.nodes[at.leaf_node[n]].level));
  h->dsleaf = upload(h, sl, st);
  panel_projections(h->spec, &C2F, &F2C);
  h->dC2F = upload(h, C2F, st);
  h->dF2C = upload(h, F2C, st);
  h->dev_err = (unsigned*)dalloc(h, sizeof(unsigned) * 4);
  if (!h->dD || !h->dDD || !h->dIi || !h->dprow || !h->dP || !h->dQi || !h->dQP || !h->diidx || !h->dsleaf ||
      !h->dC2F || !h->dF2C || !h->dev_err)
    return HPS_ERR_OOM;
  HPS_CUDA(cudaMemsetAsync(h->dev_err, 0, sizeof(unsigned) * 4, st));
  LeafConsts& k = h->lc;
  k = LeafConsts{};
  k.dim = 3; k.p = p; k.npts = (int)h->npts; k.nb = nb; k.s = 1.0; k.eta = 0.0;
  k.D = h->dD; k.DD = h->dDD; k.ni = ni; k.ne = h->dref.ne; k.nown = 0;
  k.Ii = h->dIi; k.prow = h->dprow; k.P = h->dP; k.iidx = h->diidx; k.sleaf = h->dsleaf;

  // ---- staged inputs
  std::vector<void*> tmpbufs;
  auto stage = [&](const void* src, size_t bytes) -> const void* {
    if (!src || is_device_ptr(src)) return src;
    void* d = dalloc(h, bytes, &tmpbufs);
    if (!d) return nullptr;
    if (cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return nullptr;
    return d;
  };
  const size_t cbytes = (size_t)nl * h->npts * sizeof(double);
  Coeffs co{};
  co.a = (const double*)stage(cf->a, cbytes);
  for (int a = 0; a < 3; ++a) co.b[a] = (const double*)stage(cf->b[a], cbytes);
  co.c = (const double*)stage(cf->c, cbytes);
  const T* f = (const T*)stage(f_in, cbytes);
  if ((cf->a && !co.a) || (cf->c && !co.c) || (f_in && !f)) return HPS_ERR_OOM;
  for (int a = 0; a < 3; ++a)
    if (cf->b[a] && !co.b[a]) return HPS_ERR_OOM;

  // ---- leaf stage
  h->leafA = dalloc(h, (size_t)nl * ni * ni * sizeof(T));
  h->leafX = dalloc(h, (size_t)nl * ni * (nb + 1) * sizeof(T));
  h->leafTH = dalloc(h, (size_t)nl * nb * (nb + 1) * sizeof(T));
  h->leaf_ipiv = (int*)dalloc(h, (size_t)nl * ni * sizeof(int));
  h->leaf_perm = (int*)dalloc(h, (size_t)nl * ni * sizeof(int));
  h->leaf_info = (int*)dalloc(h, (size_t)nl * sizeof(int));
  h->scratch = dalloc(h, scratch_R * sizeof(T));
  h->aproj_tmp = dalloc(h, std::max<size_t>(tmp, 16) * sizeof(T));
  if (!h->leafA || !h->leafX || !h->leafTH || !h->leaf_ipiv || !h->leaf_perm || !h->leaf_info || !h->scratch ||
      !h->aproj_tmp)
    return HPS_ERR_OOM;
  HPS_CUDA(cudaMemsetAsync(h->leaf_info, 0, (size_t)nl * sizeof(int), st));
  T* RHS = (T*)h->scratch;
  HPS_CUDA(leaf_dtn_assemble(k, nl, co, f, (T*)h->leafA, RHS, st, pf));
  h->leaf_G = lu_group_size<T>(ni, (int)nl, h->num_sms);
  if (h->leaf_G > 1) {
    h->leaf_luw.bars = (unsigned*)dalloc(h, sizeof(unsigned) * 2 * nl);
    h->leaf_luw.pub_bytes = lu_pub_bytes<T>(ni, (int)nl, h->leaf_G);
    h->leaf_luw.pub = dalloc(h, h->leaf_luw.pub_bytes);
    if (!h->leaf_luw.bars || !h->leaf_luw.pub) return HPS_ERR_OOM;
    HPS_CUDA(cudaMemsetAsync(h->leaf_luw.bars, 0, sizeof(unsigned) * 2 * nl, st));
  }
  BOp<T> LA = bop<T>((T*)h->leafA, (int64_t)ni * ni, ni);
  HPS_CUDA(getrf<T>(LA, ni, (int)nl, h->leaf_ipiv, h->leaf_perm, h->leaf_info, h->dev_err, h->leaf_G, h->leaf_luw,
                    st, pf));
  BOp<T> LX = bop<T>((T*)h->leafX, (int64_t)ni * (nb + 1), ni);
  HPS_CUDA(permute_rows<T>(bop<T>(RHS, (int64_t)ni * (nb + 1), ni), LX, h->leaf_perm, ni, nb + 1, (int)nl, st, pf));
  HPS_CUDA(getrs_inplace<T>(LA, ni, LX, nb + 1, (int)nl, st, pf));
  HPS_CUDA(leaf_dtn_init_T(h->dQP, nb, 1.0, nl, (T*)h->leafTH, st, pf));
  {
    GemmArgs<T> g;
    g.M = nb; g.N = nb + 1; g.K = ni; g.batch = (int)nl;
    g.A = bop<T>(h->dQi, 0, nb);
    g.B = LX;
    g.C = bop<T>((T*)h->leafTH, (int64_t)nb * (nb + 1), nb);
    g.alpha = -1.0; g.beta = 1.0;
    HPS_CUDA(gemm<T>(g, st, pf));
  }
  // T = s (QP - Q_i X) per leaf size
  HPS_CUDA(scale_blocks<T>((T*)h->leafTH, (int64_t)nb * (nb + 1), h->dsleaf, nl, st, pf));

  // ---- nonuniform merges, level by level from the deepest.  Per merge: the
  // children's [T | h] projected onto the coarsened interfaces and gathered
  // into D, [C | h_int] and [A | h_ext]; per group of equal-size merges of
  // the level: LU(D) and X = D^{-1}[C | h_int] as batched calls; per merge:
  // [T | h] = [A | h_ext] - B X.
  h->node_merge.assign(at.nodes.size(), -1);
  h->am.resize(at.plans.size());
  h->ag.clear();
  for (size_t mi = 0; mi < at.plans.size(); ++mi) h->node_merge[at.plans[mi].node] = (int)mi;
  std::vector<T*> Rof(at.plans.size(), nullptr);
  // per level, every (merge, child) projection, fill and gather runs as one
  // grouped launch per step (task tables uploaded per level)
  std::vector<std::vector<ProjTask<T>>> keep_pc, keep_pr;
  std::vector<std::vector<ZeroTask<T>>> keep_z;
  std::vector<std::vector<GatherTask<T>>> keep_g;
  for (size_t i0 = 0; i0 < at.plans.size();) {
    const int lev = at.nodes[at.plans[i0].node].level;
    size_t i1 = i0;
    while (i1 < at.plans.size() && at.nodes[at.plans[i1].node].level == lev) ++i1;
    size_t roff = 0;
    keep_pc.emplace_back();
    keep_pr.emplace_back();
    keep_z.emplace_back();
    keep_g.emplace_back();
    std::vector<ProjTask<T>>& tpc = keep_pc.back();
    std::vector<ProjTask<T>>& tpr = keep_pr.back();
    std::vector<ZeroTask<T>>& tz = keep_z.back();
    std::vector<GatherTask<T>>& tg = keep_g.back();
    int64_t tot_pc = 0, tot_pr = 0, tot_z = 0, tot_g = 0;
    size_t tmp_elems = 0;                      // level temporary: projected columns of every child
    std::vector<size_t> tmp_off;
    for (size_t mi = i0; mi < i1; ++mi) {
      const MergePlanA& pl = at.plans[mi];
      AMergeDev& M = h->am[mi];
      M.node = pl.node;
      M.n_ext = pl.n_ext;
      M.n_int = pl.n_int;
      const int ne = pl.n_ext, nI = pl.n_int;
      M.TP = dalloc(h, (size_t)ne * (ne + 1) * sizeof(T));
      M.D = dalloc(h, (size_t)nI * nI * sizeof(T));
      M.X = dalloc(h, (size_t)nI * (ne + 1) * sizeof(T));
      if (!M.TP || !M.D || !M.X) return HPS_ERR_OOM;
      const ANode& nd = at.nodes[pl.node];
      // project every child onto the coarsened interfaces
      for (int c = 0; c < 8; ++c) {
        const ChildProj& cp = pl.ch[c];
        AChildDev& CD = M.ch[c];
        std::vector<int4> src4(cp.np);
        for (int i = 0; i < cp.np; ++i) src4[i] = make_int4(cp.src[i][0], cp.src[i][1], cp.src[i][2], cp.src[i][3]);
        CD.pj.n = cp.n;
        CD.pj.np = cp.np;
        CD.pj.q2 = q2;
        CD.pj.kind = up_vec(h, cp.kind, st);
        CD.pj.u = up_vec(h, cp.u, st);
        CD.pj.src = up_vec(h, src4, st);
        CD.pj.bcopy = up_vec(h, cp.back_copy, st);
        CD.pj.bbase = up_vec(h, cp.back_base, st);
        CD.pj.bquad = up_vec(h, cp.back_quad, st);
        CD.pj.bt = up_vec(h, cp.back_t, st);
        CD.ext = up_vec(h, cp.ext, st);
        CD.var = up_vec(h, cp.var, st);
        CD.barow = up_vec(h, cp.b_arow, st);
        CD.bacol = up_vec(h, cp.b_acol, st);
        CD.bbrow = up_vec(h, cp.b_brow, st);
        CD.bcrow = up_vec(h, cp.b_crow, st);
        CD.ne_c = (int)cp.b_arow.size();
        CD.ni_c = (int)cp.b_acol.size();
        CD.Tp = dalloc(h, (size_t)cp.np * (cp.np + 1) * sizeof(T));
        if (!CD.pj.kind || !CD.pj.u || !CD.pj.src || !CD.pj.bcopy || !CD.pj.bbase || !CD.pj.bquad || !CD.pj.bt ||
            !CD.ext || !CD.var || !CD.barow || !CD.bacol || !CD.bbrow || !CD.bcrow || !CD.Tp)
          return HPS_ERR_OOM;
        int n = 0, ld = 0;
        const T* Tc = child_T(h, nd.child[c], &n, &ld);
        ProjTask<T> pc{};
        pc.src = Tc; pc.ld_src = ld; pc.nrc = n; pc.pj = CD.pj; pc.out = nullptr; pc.ld_out = n;
        pc.elem0 = tot_pc;
        tot_pc += (int64_t)n * (cp.np + 1);
        tmp_off.push_back(tmp_elems);
        tmp_elems += (size_t)n * (cp.np + 1);
        tpc.push_back(pc);
        ProjTask<T> pr{};
        pr.src = nullptr; pr.ld_src = n; pr.nrc = cp.np + 1; pr.pj = CD.pj; pr.out = (T*)CD.Tp; pr.ld_out = cp.np;
        pr.elem0 = tot_pr;
        tot_pr += (int64_t)cp.np * (cp.np + 1);
        tpr.push_back(pr);
      }
      T* R = (T*)h->scratch + roff;
      Rof[mi] = R;
      roff += (size_t)nI * (ne + 1);
      const std::pair<T*, int64_t> zs[3] = {{(T*)M.D, (int64_t)nI * nI}, {R, (int64_t)nI * (ne + 1)},
                                            {(T*)M.TP, (int64_t)ne * (ne + 1)}};
      for (const auto& z : zs) {
        tz.push_back(ZeroTask<T>{z.first, z.second, tot_z});
        tot_z += z.second;
      }
      for (int c = 0; c < 8; ++c) {
        const AChildDev& CD = M.ch[c];
        GatherTask<T> gt{};
        gt.Tc = (const T*)CD.Tp; gt.nbc = CD.pj.np; gt.n_ext = ne; gt.n_int = nI;
        gt.ext = CD.ext; gt.var = CD.var; gt.D = (T*)M.D; gt.R = R; gt.TP = (T*)M.TP;
        gt.elem0 = tot_g;
        tot_g += (int64_t)CD.pj.np * (CD.pj.np + 1);
        tg.push_back(gt);
      }
    }
    {
      // the level's temporary and task tables, then four launches
      T* tmpL = (T*)dalloc(h, std::max<size_t>(tmp_elems, 1) * sizeof(T), &tmpbufs);
      if (!tmpL) return HPS_ERR_OOM;
      for (size_t t = 0; t < tpc.size(); ++t) {
        tpc[t].out = tmpL + tmp_off[t];
        tpr[t].src = tmpL + tmp_off[t];
      }
      auto up_tasks = [&](const auto& v) -> void* {
        const size_t bytes = v.size() * sizeof(v[0]);
        void* d = dalloc(h, std::max<size_t>(bytes, 16), &tmpbufs);
        if (d && bytes && cudaMemcpyAsync(d, v.data(), bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return nullptr;
        return d;
      };
      auto* dpc = (const ProjTask<T>*)up_tasks(tpc);
      auto* dpr = (const ProjTask<T>*)up_tasks(tpr);
      auto* dz = (const ZeroTask<T>*)up_tasks(tz);
      auto* dg = (const GatherTask<T>*)up_tasks(tg);
      if (!dpc || !dpr || !dz || !dg) return HPS_ERR_OOM;
      HPS_CUDA(proj_cols_group<T>(dpc, (int)tpc.size(), tot_pc, h->dC2F, st, pf));
      HPS_CUDA(proj_rows_group<T>(dpr, (int)tpr.size(), tot_pr, h->dF2C, st, pf));
      HPS_CUDA(zero_group<T>(dz, (int)tz.size(), tot_z, st, pf));
      HPS_CUDA(merge_gather_group<T>(dg, (int)tg.size(), tot_g, st, pf));
    }
    // groups of equal sizes within the level, in first-appearance order
    std::vector<std::pair<std::pair<int, int>, std::vector<int>>> groups;
    for (size_t mi = i0; mi < i1; ++mi) {
      const std::pair<int, int> key(at.plans[mi].n_int, at.plans[mi].n_ext);
      size_t gi = 0;
      while (gi < groups.size() && groups[gi].first != key) ++gi;
      if (gi == groups.size()) groups.push_back({key, {}});
      groups[gi].second.push_back((int)mi);
    }
    for (auto& gr : groups) {
      AGroup A;
      A.level = lev;
      A.n_int = gr.first.first;
      A.n_ext = gr.first.second;
      A.members = gr.second;
      const int nI = A.n_int, ne = A.n_ext, nbat = (int)A.members.size();
      A.ipiv = (int*)dalloc(h, (size_t)nbat * nI * sizeof(int));
      A.perm = (int*)dalloc(h, (size_t)nbat * nI * sizeof(int));
      A.info = (int*)dalloc(h, (size_t)nbat * sizeof(int));
      std::vector<T*> vD, vX, vR;
      for (int k2 = 0; k2 < nbat; ++k2) {
        AMergeDev& M = h->am[(size_t)A.members[k2]];
        vD.push_back((T*)M.D);
        vX.push_back((T*)M.X);
        vR.push_back(Rof[(size_t)A.members[k2]]);
      }
      A.dD = upload(h, vD, st);
      A.dX = upload(h, vX, st);
      A.dR = upload(h, vR, st);
      if (!A.ipiv || !A.perm || !A.info || !A.dD || !A.dX || !A.dR) return HPS_ERR_OOM;
      HPS_CUDA(cudaMemsetAsync(A.info, 0, (size_t)nbat * sizeof(int), st));
      for (int k2 = 0; k2 < nbat; ++k2) {
        AMergeDev& M = h->am[(size_t)A.members[k2]];
        M.ipiv = A.ipiv + (size_t)k2 * nI;
        M.perm = A.perm + (size_t)k2 * nI;
        M.info = A.info + k2;
      }
      A.G = lu_group_size<T>(nI, nbat, h->num_sms);
      if (A.G > 1) {
        A.luw.bars = (unsigned*)dalloc(h, sizeof(unsigned) * 2 * nbat);
        A.luw.pub_bytes = lu_pub_bytes<T>(nI, nbat, A.G);
        A.luw.pub = dalloc(h, A.luw.pub_bytes);
        if (!A.luw.bars || !A.luw.pub) return HPS_ERR_OOM;
        HPS_CUDA(cudaMemsetAsync(A.luw.bars, 0, sizeof(unsigned) * 2 * nbat, st));
      }
      BOp<T> DD = bopp<T>(A.dD, nI);
      BOp<T> XX = bopp<T>(A.dX, nI);
      HPS_CUDA(getrf<T>(DD, nI, nbat, A.ipiv, A.perm, A.info, h->dev_err, A.G, A.luw, st, pf));
      AMergeDev& M0 = h->am[(size_t)A.members[0]];
      if (nbat == 1 && M0.node == 0 && h->opts.lazy_root && !h->opts.want_root_map) {
        // lazy root: keep [C | h_int] (in X's storage) and D's factors
        M0.lazy = true;
        HPS_CUDA(cudaMemcpyAsync(M0.X, Rof[(size_t)A.members[0]], (size_t)nI * (ne + 1) * sizeof(T),
                                 cudaMemcpyDeviceToDevice, st));
        const int nf = (nI + 31) / 32;
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
      } else {
        HPS_CUDA(permute_rows<T>(bopp<T>(A.dR, nI), XX, A.perm, nI, ne + 1, nbat, st, pf));
        HPS_CUDA(getrs_inplace<T>(DD, nI, XX, ne + 1, nbat, st, pf));
      }
      std::vector<T*> vTP;
      for (int mi : A.members) vTP.push_back((T*)h->am[(size_t)mi].TP);
      A.dTP = upload(h, vTP, st);
      if (!A.dTP) return HPS_ERR_OOM;
      for (int c = 0; c < 8; ++c) {
        AGroup::ChildBatch& cb = A.cb[c];
        const ChildProj& c0 = at.plans[(size_t)A.members[0]].ch[c];
        cb.ok = nbat > 1;
        for (int mi : A.members) {
          const ChildProj& cp = at.plans[(size_t)mi].ch[c];
          if (cp.b_arow.size() != c0.b_arow.size() || cp.b_acol.size() != c0.b_acol.size() || cp.np != c0.np)
            cb.ok = false;
        }
        if (!cb.ok) continue;
        cb.ne_c = (int)c0.b_arow.size();
        cb.ni_c = (int)c0.b_acol.size();
        cb.np = c0.np;
        std::vector<int> ar, ac, br, cr;
        std::vector<T*> tp;
        for (int mi : A.members) {
          const ChildProj& cp = at.plans[(size_t)mi].ch[c];
          ar.insert(ar.end(), cp.b_arow.begin(), cp.b_arow.end());
          ac.insert(ac.end(), cp.b_acol.begin(), cp.b_acol.end());
          br.insert(br.end(), cp.b_brow.begin(), cp.b_brow.end());
          cr.insert(cr.end(), cp.b_crow.begin(), cp.b_crow.end());
          tp.push_back((T*)h->am[(size_t)mi].ch[c].Tp);
        }
        cb.barow = upload(h, ar, st);
        cb.bacol = upload(h, ac, st);
        cb.bbrow = upload(h, br, st);
        cb.bcrow = upload(h, cr, st);
        cb.dTp = upload(h, tp, st);
        if (!cb.barow || !cb.bacol || !cb.bbrow || !cb.bcrow || !cb.dTp) return HPS_ERR_OOM;
      }
      h->ag.push_back(std::move(A));
    }
    // [T | h] = [A | h_ext] - B X, one product per child position of a group
    for (size_t gi = h->ag.size() - groups.size(); gi < h->ag.size(); ++gi) {
      const AGroup& A = h->ag[gi];
      HPS_TRY(group_b_products(h, A, A.dX, A.n_ext + 1, A.dTP, true, st, pf));
    }
    i0 = i1;
  }
  HPS_CUDA(cudaStreamSynchronize(st));
  for (void* tb : tmpbufs) dev_free(tb, st);
  unsigned derr = 0;
  HPS_CUDA(cudaMemcpy(&derr, h->dev_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (derr & DEV_ERR_TIMEOUT) return HPS_ERR_TIMEOUT;
  std::vector<int> info(nl);
  HPS_CUDA(cudaMemcpy(info.data(), h->leaf_info, nl * sizeof(int), cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < nl; ++i)
    if (info[i]) { h->err_node = i; return HPS_ERR_SINGULAR; }
  for (size_t mi = 0; mi < h->am.size(); ++mi) {
    int v = 0;
    HPS_CUDA(cudaMemcpy(&v, h->am[mi].info, sizeof(int), cudaMemcpyDeviceToHost));
    if (v) { h->err_node = nl + (int64_t)mi; return HPS_ERR_SINGULAR; }
  }
  return HPS_OK;
}

static hps_status adaptive_ws(hps_handle* h, int nrhs) {
  using T = double;
  if (h->ws_nrhs >= nrhs) return HPS_OK;
  // the call has ordered h->last after the handle's earlier work
  for (void* pp : h->ws_allocs) dev_free(pp, h->last);
  h->ws_allocs.clear();
  h->bytes -= h->ws_bytes;
  const int64_t before = h->bytes;
  const size_t es = sizeof(T);
  auto A = [&](size_t bytes) { return dalloc(h, bytes, &h->ws_allocs); };
  h->ws_xf = A((size_t)h->nl * h->xrows_leaf * nrhs * es);
  h->ws_hleaf = A((size_t)h->nl * h->nb * nrhs * es);
  h->ws_gleaf = A((size_t)h->nl * h->nb * nrhs * es);
  h->ws_g = A((size_t)h->nroot * nrhs * es);
  h->ws_f = A((size_t)h->nl * h->npts * nrhs * es);
  h->ws_u = A((size_t)h->nl * h->npts * nrhs * es);
  h->ws_rhs = A((size_t)h->nl * h->xrows_leaf * nrhs * es);
  void* vt = A((size_t)std::max(h->max_np, 1) * nrhs * es);
  if (!h->ws_xf || !h->ws_hleaf || !h->ws_gleaf || !h->ws_g || !h->ws_f || !h->ws_u || !h->ws_rhs || !vt)
    return HPS_ERR_OOM;
  h->ws_vtmp = vt;
  for (AMergeDev& M : h->am) {
    M.r = A((size_t)M.n_int * nrhs * es);
    M.x = A((size_t)M.n_int * nrhs * es);
    M.hp = A((size_t)M.n_ext * nrhs * es);
    M.gint = A((size_t)M.n_int * nrhs * es);
    M.g = A((size_t)M.n_ext * nrhs * es);
    if (!M.r || !M.x || !M.hp || !M.gint || !M.g) return HPS_ERR_OOM;
  }
  // pointer arrays of the batched group solves
  for (AGroup& G : h->ag) {
    std::vector<T*> vr, vx, vh;
    for (int mi : G.members) {
      vr.push_back((T*)h->am[(size_t)mi].r);
      vx.push_back((T*)h->am[(size_t)mi].x);
      vh.push_back((T*)h->am[(size_t)mi].hp);
    }
    const size_t pb = vr.size() * sizeof(T*);
    G.dr = (T**)A(pb);
    G.dx = (T**)A(pb);
    G.dhp = (T**)A(pb);
    if (!G.dr || !G.dx || !G.dhp) return HPS_ERR_OOM;
    if (cudaMemcpy(G.dr, vr.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.dx, vx.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.dhp, vh.data(), pb, cudaMemcpyHostToDevice) != cudaSuccess)
      return HPS_ERR_CUDA;
  }
  // task tables of the grouped solve passes, level by level (deepest first)
  {
    const ATree& at = h->at;
    h->alev.clear();
    for (size_t mi = 0; mi < h->am.size(); ++mi) {
      const int lev = at.nodes[h->am[mi].node].level;
      if (h->alev.empty() || at.nodes[h->am[(size_t)h->alev.back().merges[0]].node].level != lev)
        h->alev.emplace_back();
      h->alev.back().merges.push_back((int)mi);
    }
    size_t vtot = 0;
    for (const AMergeDev& M : h->am)
      for (int c = 0; c < 8; ++c) vtot += (size_t)M.ch[c].pj.np * nrhs;
    T* vall = (T*)A(std::max<size_t>(vtot, 1) * es);
    if (!vall) return HPS_ERR_OOM;
    size_t voff = 0;
    for (ASolveLevel& Lv : h->alev) {
      std::vector<ZeroTask<T>> zr;
      std::vector<ProjTask<T>> pr, un;
      std::vector<ChildTask<T>> gh, dc;
      std::vector<GintTask<T>> gi;
      for (int mi : Lv.merges) {
        AMergeDev& M = h->am[(size_t)mi];
        const ANode& nd = at.nodes[M.node];
        zr.push_back(ZeroTask<T>{(T*)M.r, (int64_t)M.n_int * nrhs, Lv.tzr});
        Lv.tzr += (int64_t)M.n_int * nrhs;
        if (!M.lazy) {
          GintTask<T> t{};
          t.X = (const T*)M.X; t.xp = (const T*)M.x; t.gpar = (const T*)M.g; t.gint = (T*)M.gint;
          t.n_ext = M.n_ext; t.n_int = M.n_int; t.nrhs = nrhs; t.tile0 = Lv.tgi;
          Lv.tgi += (int64_t)((M.n_int + 31) / 32) * nrhs;
          gi.push_back(t);
        }
        for (int c = 0; c < 8; ++c) {
          const AChildDev& CD = M.ch[c];
          const int np = CD.pj.np;
          T* v = vall + voff;
          voff += (size_t)np * nrhs;
          const ANode& K = at.nodes[nd.child[c]];
          T *hc, *gc;
          int ld;
          if (K.leaf >= 0) {
            hc = (T*)h->ws_hleaf + (int64_t)K.leaf * h->nb * nrhs;
            gc = (T*)h->ws_gleaf + (int64_t)K.leaf * h->nb * nrhs;
            ld = h->nb;
          } else {
            AMergeDev& C2 = h->am[(size_t)h->node_merge[nd.child[c]]];
            hc = (T*)C2.hp;
            gc = (T*)C2.g;
            ld = C2.n_ext;
          }
          ProjTask<T> p{};
          p.src = hc; p.ld_src = ld; p.nrc = nrhs; p.pj = CD.pj; p.out = v; p.ld_out = np; p.elem0 = Lv.tpr;
          Lv.tpr += (int64_t)np * nrhs;
          pr.push_back(p);
          ChildTask<T> g2{};
          g2.gint = v; g2.r = (T*)M.r; g2.hp = (T*)M.hp; g2.nbc = np; g2.n_ext = M.n_ext; g2.n_int = M.n_int;
          g2.nrhs = nrhs; g2.ext = CD.ext; g2.var = CD.var; g2.elem0 = Lv.tgh;
          Lv.tgh += (int64_t)np * nrhs;
          gh.push_back(g2);
          ChildTask<T> d{};
          d.gpar = (const T*)M.g; d.gint = (T*)M.gint; d.out = v; d.nbc = np; d.n_ext = M.n_ext;
          d.n_int = M.n_int; d.nrhs = nrhs; d.ext = CD.ext; d.var = CD.var; d.elem0 = Lv.tdc;
          Lv.tdc += (int64_t)np * nrhs;
          dc.push_back(d);
          ProjTask<T> q{};
          q.src = v; q.ld_src = np; q.nrc = nrhs; q.pj = CD.pj; q.out = gc; q.ld_out = ld; q.elem0 = Lv.tun;
          Lv.tun += (int64_t)CD.pj.n * nrhs;
          un.push_back(q);
        }
      }
      auto up = [&](const auto& vec, auto** dst, int* cnt) -> bool {
        const size_t bytes = std::max<size_t>(vec.size() * sizeof(vec[0]), 16);
        void* d = A(bytes);
        if (!d) return false;
        if (!vec.empty() && cudaMemcpy(d, vec.data(), vec.size() * sizeof(vec[0]), cudaMemcpyHostToDevice) != cudaSuccess)
          return false;
        *dst = (std::remove_reference_t<decltype(**dst)>*)d;
        *cnt = (int)vec.size();
        return true;
      };
      if (!up(zr, &Lv.zr, &Lv.nzr) || !up(pr, &Lv.pr, &Lv.npr) || !up(gh, &Lv.gh, &Lv.ngh) ||
          !up(gi, &Lv.gi, &Lv.ngi) || !up(dc, &Lv.dc, &Lv.ndc) || !up(un, &Lv.un, &Lv.nun))
        return HPS_ERR_OOM;
    }
  }
  h->ws_bytes = h->bytes - before;
  h->ws_nrhs = nrhs;
  return HPS_OK;
}

hps_status adaptive_solve(hps_handle* h, int nrhs, const void* g_in, const void* f_in, void* u_out,
                          cudaStream_t st) {
  using T = double;
  if (h->trsv_err_host && *(volatile int*)h->trsv_err_host) return HPS_ERR_TIMEOUT;
  hps_status rs = adaptive_ws(h, nrhs);
  if (rs != HPS_OK) return rs;
  Prof* pf = &h->prof;
  pf->reset();
  pf->on = h->opts.profile != 0;
  const ATree& at = h->at;
  const int64_t nl = h->nl;
  const int nb = h->nb, ni = h->dref.ni;
  const T* g = (const T*)g_in;
  if (!is_device_ptr(g_in)) {
    HPS_CUDA(cudaMemcpyAsync(h->ws_g, g_in, (size_t)h->nroot * nrhs * sizeof(T), cudaMemcpyHostToDevice, st));
    g = (const T*)h->ws_g;
  }
  const T* f = (const T*)f_in;
  if (f_in && !is_device_ptr(f_in)) {
    HPS_CUDA(cudaMemcpyAsync(h->ws_f, f_in, (size_t)nl * h->npts * nrhs * sizeof(T), cudaMemcpyHostToDevice, st));
    f = (const T*)h->ws_f;
  }
  const bool host_u = !is_device_ptr(u_out);
  T* u = host_u ? (T*)h->ws_u : (T*)u_out;
  const bool newf = f != nullptr;
  T* vt = (T*)h->ws_vtmp;

  if (newf) {
    T* xf = (T*)h->ws_xf;
    T* tmp = (T*)h->ws_rhs;
    HPS_CUDA(leaf_particular_rhs<T>(h->lc, nl, nrhs, f, tmp, false, st, pf));
    BOp<T> LA = bop<T>((T*)h->leafA, (int64_t)ni * ni, ni);
    BOp<T> XF = bop<T>(xf, (int64_t)ni * nrhs, ni);
    HPS_CUDA(permute_rows<T>(bop<T>(tmp, (int64_t)ni * nrhs, ni), XF, h->leaf_perm, ni, nrhs, (int)nl, st, pf));
    HPS_CUDA(getrs_inplace<T>(LA, ni, XF, nrhs, (int)nl, st, pf));
    GemmArgs<T> gl;
    gl.M = nb; gl.N = nrhs; gl.K = ni; gl.batch = (int)nl;
    gl.A = bop<T>(h->dQi, 0, nb);
    gl.B = XF;
    gl.C = bop<T>((T*)h->ws_hleaf, (int64_t)nb * nrhs, nb);
    gl.alpha = -1.0; gl.beta = 0.0;
    HPS_CUDA(gemm<T>(gl, st, pf));
    HPS_CUDA(scale_blocks<T>((T*)h->ws_hleaf, (int64_t)nb * nrhs, h->dsleaf, nl, st, pf));
    // level by level: gathers of every merge of the level, one batched
    // D^{-1} per group of equal sizes, then the B x products
    size_t lv = 0;
    for (size_t g0 = 0; g0 < h->ag.size();) {
      size_t g1 = g0;
      while (g1 < h->ag.size() && h->ag[g1].level == h->ag[g0].level) ++g1;
      // every merge of the level: zero r, project each child's h, gather it
      const ASolveLevel& L = h->alev[lv++];
      HPS_CUDA(zero_group<T>(L.zr, L.nzr, L.tzr, st, pf));
      HPS_CUDA(proj_rows_group<T>(L.pr, L.npr, L.tpr, h->dF2C, st, pf));
      HPS_CUDA(gather_h_group<T>(L.gh, L.ngh, L.tgh, st, pf));
      for (size_t gi = g0; gi < g1; ++gi) {
        const AGroup& G = h->ag[gi];
        const int nbat = (int)G.members.size();
        if (h->am[(size_t)G.members[0]].lazy) continue;  // the root's D^{-1} runs in the downward pass
        BOp<T> XB = bopp<T>(G.dx, G.n_int);
        HPS_CUDA(permute_rows<T>(bopp<T>(G.dr, G.n_int), XB, G.perm, G.n_int, nrhs, nbat, st, pf));
        HPS_CUDA(getrs_inplace<T>(bopp<T>(G.dD, G.n_int), G.n_int, XB, nrhs, nbat, st, pf));
      }
      for (size_t gi = g0; gi < g1; ++gi) {
        const AGroup& G = h->ag[gi];
        HPS_TRY(group_b_products(h, G, G.dx, nrhs, G.dhp, false, st, pf));
      }
      g0 = g1;
    }
  }
  // downward pass, root level first: the root's data is copied into its own
  // workspace so that every level's task tables refer to fixed buffers
  if (!h->am.empty()) {
    AMergeDev& R0 = h->am[(size_t)h->node_merge[0]];
    HPS_CUDA(cudaMemcpyAsync(R0.g, g, (size_t)R0.n_ext * nrhs * sizeof(T), cudaMemcpyDeviceToDevice, st));
  }
  for (size_t li = h->alev.size(); li-- > 0;) {
    const ASolveLevel& L = h->alev[li];
    for (int mi : L.merges) {
      AMergeDev& M = h->am[(size_t)mi];
      if (!M.lazy) continue;
      const T* gpar = (const T*)M.g;
      // X holds [C | h_int]: t = -(C g + h), then g_int = D^{-1} t
      HPS_CUDA(down_gint<T>((const T*)M.X, newf ? (const T*)M.r : nullptr, gpar, 1, M.n_ext, M.n_int, nrhs,
                            (T*)M.x, st, pf));
      BOp<T> GI = bop<T>((T*)M.gint, 0, M.n_int);
      HPS_CUDA(permute_rows<T>(bop<T>((T*)M.x, 0, M.n_int), GI, M.perm, M.n_int, nrhs, 1, st, pf));
      if (trsv_flags_applicable<T>(M.n_int, nrhs, 1, h->trsv))
        HPS_CUDA(getrs_flags<T>((const T*)M.D, M.n_int, M.n_int, (T*)M.gint, M.n_int, nrhs, h->trsv, st, pf));
      else
        HPS_CUDA(getrs_inplace<T>(bop<T>((T*)M.D, 0, M.n_int), M.n_int, GI, nrhs, 1, st, pf));
    }
    // the level's other merges, their children's data and its unprojection
    HPS_CUDA(gint_group<T>(L.gi, L.ngi, L.tgi, newf ? 1 : 0, st, pf));
    HPS_CUDA(down_children_group<T>(L.dc, L.ndc, L.tdc, st, pf));
    HPS_CUDA(unproject_group<T>(L.un, L.nun, L.tun, h->dC2F, st, pf));
  }
  const T* gleaf = h->am.empty() ? g : (const T*)h->ws_gleaf;
  HPS_CUDA(leaf_output<T>(h->lc, nl, nrhs, (const T*)h->leafX, newf ? (const T*)h->ws_xf : nullptr, gleaf, u, false,
                          st, pf));
  if (host_u) {
    HPS_CUDA(cudaMemcpyAsync(u_out, u, (size_t)nl * h->npts * nrhs * sizeof(T), cudaMemcpyDeviceToHost, st));
    HPS_CUDA(cudaStreamSynchronize(st));
  }
  return HPS_OK;
}

// ---------------------------------------------------------------- refine ----

namespace {

// p Chebyshev values on [-1, 1] -> the two children's Chebyshev nodes
// ([-1, 0] then [0, 1]): 2p x p, row-major.
std::vector<double> child_interp(const Spectral1D& s) {
  const int p = s.p;
  std::vector<double> w(p), M((size_t)2 * p * p, 0.0);
  for (int j = 0; j < p; ++j) {
    w[j] = 1.0;
    for (int k = 0; k < p; ++k)
      if (k != j) w[j] *= (s.xc[j] - s.xc[k]);
    w[j] = 1.0 / w[j];
  }
  for (int i = 0; i < 2 * p; ++i) {
    const double t = (i < p) ? 0.5 * (s.xc[i] - 1.0) : 0.5 * (s.xc[i - p] + 1.0);
    int hit = -1;
    for (int j = 0; j < p; ++j)
      if (t == s.xc[j]) hit = j;
    if (hit >= 0) { M[(size_t)i * p + hit] = 1.0; continue; }
    double den = 0.0;
    for (int j = 0; j < p; ++j) den += w[j] / (t - s.xc[j]);
    for (int j = 0; j < p; ++j) M[(size_t)i * p + j] = (w[j] / (t - s.xc[j])) / den;
  }
  return M;
}

void leaf_points(const double* lo, double side, int level, const int64_t* ix, const Spectral1D& s, double* out) {
  const int p = s.p;
  const double h = side / (double)((int64_t)1 << level);
  for (int node = 0; node < p * p * p; ++node) {
    const int c[3] = {node % p, (node / p) % p, node / (p * p)};
    for (int a = 0; a < 3; ++a) out[(size_t)node * 3 + a] = lo[a] + (ix[a] + 0.5 * (s.xc[c[a]] + 1.0)) * h;
  }
}

}  // namespace

hps_status adaptive_refine(const double* lo, const double* hi, int p, double eps, int min_depth, int max_depth,
                           int n_fn, const hps_eval_fn* fns, void* const* ctxs, int64_t capacity,
                           int64_t* n_leaves, uint64_t* morton, int8_t* level, cudaStream_t st) {
  if (!lo || !hi || p < 4 || p > 24 || !(eps > 0) || min_depth < 0 || max_depth < min_depth || max_depth > 10 ||
      n_fn < 1 || !fns || !n_leaves)
    return HPS_ERR_INVALID;
  const double side = hi[0] - lo[0];
  if (!(side > 0)) return HPS_ERR_INVALID;
  for (int a = 1; a < 3; ++a)
    if (!(std::fabs((hi[a] - lo[a]) - side) <= 1e-12 * side)) return HPS_ERR_INVALID;
  const Spectral1D s = make_spectral(p, p - 2);
  const std::vector<double> I1 = child_interp(s);
  const int npts = p * p * p;
  using Leaf = std::pair<int, std::array<int64_t, 3>>;
  std::vector<Leaf> cand, fin;
  const int64_t n1 = (int64_t)1 << min_depth;
  for (int64_t z = 0; z < n1; ++z)
    for (int64_t y = 0; y < n1; ++y)
      for (int64_t x = 0; x < n1; ++x) cand.push_back({min_depth, {x, y, z}});
  std::vector<double> norms(n_fn, 0.0);
  double* dI1 = nullptr;
  double *d0 = nullptr, *d1 = nullptr, *derr = nullptr;
  size_t cap_leaves = 0;
  auto release = [&]() {
    cudaFree(dI1); cudaFree(d0); cudaFree(d1); cudaFree(derr);
    dI1 = d0 = d1 = derr = nullptr;
  };
  if (cudaMalloc(&dI1, I1.size() * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return HPS_ERR_OOM; }
  if (cudaMemcpy(dI1, I1.data(), I1.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    release();
    return HPS_ERR_CUDA;
  }
  while (!cand.empty()) {
    if (cand[0].first >= max_depth) {
      fin.insert(fin.end(), cand.begin(), cand.end());
      break;
    }
    const size_t nc = cand.size();
    std::vector<double> x0(nc * npts * 3), x1(nc * 8 * npts * 3);
    for (size_t n = 0; n < nc; ++n) {
      leaf_points(lo, side, cand[n].first, cand[n].second.data(), s, &x0[n * npts * 3]);
      for (int c = 0; c < 8; ++c) {
        const int64_t ci[3] = {2 * cand[n].second[0] + (c & 1), 2 * cand[n].second[1] + ((c >> 1) & 1),
                               2 * cand[n].second[2] + (c >> 2)};
        leaf_points(lo, side, cand[n].first + 1, ci, s, &x1[(n * 8 + c) * npts * 3]);
      }
    }
    if (nc > cap_leaves) {
      cudaFree(d0); cudaFree(d1); cudaFree(derr);
      d0 = d1 = derr = nullptr;
      if (cudaMalloc(&d0, nc * npts * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&d1, nc * 8 * npts * sizeof(double)) != cudaSuccess ||
          cudaMalloc(&derr, nc * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        release();
        return HPS_ERR_OOM;
      }
      cap_leaves = nc;
    }
    std::vector<char> split(nc, 0);
    std::vector<std::vector<double>> errs(n_fn);
    std::vector<double> v0(nc * npts), v1(nc * 8 * npts);
    for (int k = 0; k < n_fn; ++k) {
      void* ctx = ctxs ? ctxs[k] : nullptr;
      if (fns[k](ctx, (int64_t)(nc * npts), x0.data(), v0.data()) != 0 ||
          fns[k](ctx, (int64_t)(nc * 8 * npts), x1.data(), v1.data()) != 0) {
        release();
        return HPS_ERR_INVALID;
      }
      for (double v : v0) norms[k] = std::max(norms[k], std::fabs(v));
      for (double v : v1) norms[k] = std::max(norms[k], std::fabs(v));
      errs[k].resize(nc);
      if (cudaMemcpyAsync(d0, v0.data(), v0.size() * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaMemcpyAsync(d1, v1.data(), v1.size() * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          refine_check(d0, d1, (int64_t)nc, p, dI1, derr, st) != cudaSuccess ||
          cudaMemcpyAsync(errs[k].data(), derr, nc * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        release();
        return HPS_ERR_CUDA;
      }
    }
    // the norms include every sample of this level before any decision
    for (int k = 0; k < n_fn; ++k)
      for (size_t n = 0; n < nc; ++n)
        if (norms[k] > 0.0 && errs[k][n] / norms[k] >= eps) split[n] = 1;
    std::vector<Leaf> nxt;
    for (size_t n = 0; n < nc; ++n) {
      if (!split[n]) { fin.push_back(cand[n]); continue; }
      for (int c = 0; c < 8; ++c)
        nxt.push_back({cand[n].first + 1, {2 * cand[n].second[0] + (c & 1), 2 * cand[n].second[1] + ((c >> 1) & 1),
                                           2 * cand[n].second[2] + (c >> 2)}});
    }
    cand.swap(nxt);
  }
  release();
  balance_leaves(&fin);
  *n_leaves = (int64_t)fin.size();
  if ((int64_t)fin.size() > capacity || !morton || !level) return capacity < 0 ? HPS_ERR_INVALID : HPS_OK;
  for (size_t n = 0; n < fin.size(); ++n) {
    morton[n] = morton_encode(fin[n].second.data());
    level[n] = (int8_t)fin[n].first;
  }
  return HPS_OK;
}

}  // namespace hps
