// Adaptive octree planning (Section 4.2, nonuniform merges).
#include "adaptive.h"

#include <algorithm>
#include <cmath>
#include <set>
#include <stdexcept>

namespace hps {

namespace {

const int kFaceAxis[6] = {0, 0, 1, 1, 2, 2};
const int kFaceSide[6] = {0, 1, 0, 1, 0, 1};

void tang(int axis, int* t) {
  int k = 0;
  for (int a = 0; a < 3; ++a)
    if (a != axis) t[k++] = a;
}

// depth-first order key: child digits of the coarse levels are the most
// significant
uint64_t dfs_key(int level, const int64_t* ix) {
  uint64_t key = 0;
  for (int l = 0; l < level; ++l) {
    const int sh = level - 1 - l;
    const uint64_t c = ((ix[0] >> sh) & 1) | (((ix[1] >> sh) & 1) << 1) | (((ix[2] >> sh) & 1) << 2);
    key |= c << (3 * (20 - 1 - l));
  }
  return key;
}

struct Key {
  int level;
  int64_t x, y, z;
  bool operator<(const Key& o) const {
    if (level != o.level) return level < o.level;
    if (x != o.x) return x < o.x;
    if (y != o.y) return y < o.y;
    return z < o.z;
  }
};

// Gauss--Legendre weights on [-1, 1] for nodes x: 2 / ((1 - x^2) P_q'(x)^2).
std::vector<double> gauss_weights(const std::vector<double>& x) {
  const int q = (int)x.size();
  std::vector<double> w(q);
  for (int i = 0; i < q; ++i) {
    double p0 = 1.0, p1 = x[i];
    for (int k = 2; k <= q; ++k) {
      double p2 = ((2.0 * k - 1.0) * x[i] * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    const double dp = q * (x[i] * p1 - p0) / (x[i] * x[i] - 1.0);
    w[i] = 2.0 / ((1.0 - x[i] * x[i]) * dp * dp);
  }
  return w;
}

std::vector<double> bary_interp(const std::vector<double>& s, const std::vector<double>& t) {
  const int n = (int)s.size(), m = (int)t.size();
  std::vector<double> w(n, 1.0), M((size_t)m * n, 0.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) w[j] *= (s[j] - s[k]);
  for (auto& v : w) v = 1.0 / v;
  for (int i = 0; i < m; ++i) {
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (t[i] == s[j]) hit = j;
    if (hit >= 0) { M[(size_t)i * n + hit] = 1.0; continue; }
    double den = 0.0;
    for (int j = 0; j < n; ++j) den += w[j] / (t[i] - s[j]);
    for (int j = 0; j < n; ++j) M[(size_t)i * n + j] = (w[j] / (t[i] - s[j])) / den;
  }
  return M;
}

}  // namespace

uint64_t morton_encode(const int64_t* ix) {
  uint64_t c = 0;
  for (int b = 0; b < 21; ++b)
    for (int a = 0; a < 3; ++a) c |= (uint64_t)((ix[a] >> b) & 1) << (3 * b + a);
  return c;
}

void morton_decode(uint64_t code, int level, int64_t* ix) {
  ix[0] = ix[1] = ix[2] = 0;
  for (int b = 0; b < level; ++b)
    for (int a = 0; a < 3; ++a) ix[a] |= (int64_t)((code >> (3 * b + a)) & 1) << b;
}

void sort_leaves(std::vector<std::pair<int, std::array<int64_t, 3>>>* leaves) {
  std::sort(leaves->begin(), leaves->end(), [](const auto& a, const auto& b) {
    return dfs_key(a.first, a.second.data()) < dfs_key(b.first, b.second.data());
  });
}

void balance_leaves(std::vector<std::pair<int, std::array<int64_t, 3>>>* leaves) {
  for (;;) {
    std::set<Key> leaf, internal;
    for (auto& lv : *leaves) {
      leaf.insert({lv.first, lv.second[0], lv.second[1], lv.second[2]});
      for (int l2 = lv.first - 1; l2 >= 0; --l2) {
        const int sh = lv.first - l2;
        internal.insert({l2, lv.second[0] >> sh, lv.second[1] >> sh, lv.second[2] >> sh});
      }
    }
    std::vector<size_t> split;
    for (size_t n = 0; n < leaves->size(); ++n) {
      const int lv = (*leaves)[n].first;
      const auto& ix = (*leaves)[n].second;
      const int64_t n1 = (int64_t)1 << lv;
      bool need = false;
      for (int f = 0; f < 6 && !need; ++f) {
        int64_t nb[3] = {ix[0], ix[1], ix[2]};
        const int a = kFaceAxis[f];
        nb[a] += kFaceSide[f] ? 1 : -1;
        if (nb[a] < 0 || nb[a] >= n1) continue;
        if (!internal.count({lv, nb[0], nb[1], nb[2]})) continue;
        for (int c = 0; c < 8 && !need; ++c) {
          int64_t ci[3] = {2 * nb[0] + (c & 1), 2 * nb[1] + ((c >> 1) & 1), 2 * nb[2] + (c >> 2)};
          const bool touching = (ci[a] & 1) == (kFaceSide[f] ? 0 : 1);
          if (touching && internal.count({lv + 1, ci[0], ci[1], ci[2]})) need = true;
        }
      }
      if (need) split.push_back(n);
    }
    if (split.empty()) break;
    std::vector<std::pair<int, std::array<int64_t, 3>>> out;
    std::vector<char> mark(leaves->size(), 0);
    for (size_t s : split) mark[s] = 1;
    for (size_t n = 0; n < leaves->size(); ++n) {
      const auto& lf = (*leaves)[n];
      if (!mark[n]) { out.push_back(lf); continue; }
      for (int c = 0; c < 8; ++c)
        out.push_back({lf.first + 1, {2 * lf.second[0] + (c & 1), 2 * lf.second[1] + ((c >> 1) & 1),
                                      2 * lf.second[2] + (c >> 2)}});
    }
    *leaves = out;
  }
  sort_leaves(leaves);
}

void panel_projections(const Spectral1D& s, std::vector<double>* C2F, std::vector<double>* F2C) {
  const int q = s.q, q2 = q * q;
  std::vector<double> xc(q), xf(2 * q);
  const std::vector<double> w = gauss_weights(s.xg);
  std::vector<double> wc(q), wf(2 * q);
  for (int i = 0; i < q; ++i) {
    xc[i] = 0.5 * (s.xg[i] + 1.0);
    wc[i] = 0.5 * w[i];
    xf[i] = 0.25 * (s.xg[i] + 1.0);
    xf[q + i] = 0.5 + 0.25 * (s.xg[i] + 1.0);
    wf[i] = wf[q + i] = 0.25 * w[i];
  }
  const std::vector<double> c2f1 = bary_interp(xc, xf);  // 2q x q row-major
  std::vector<double> f2c1((size_t)q * 2 * q);           // q x 2q row-major
  for (int i = 0; i < q; ++i)
    for (int k = 0; k < 2 * q; ++k) f2c1[(size_t)i * 2 * q + k] = wf[k] * c2f1[(size_t)k * q + i] / wc[i];
  C2F->assign((size_t)4 * q2 * q2, 0.0);
  F2C->assign((size_t)q2 * 4 * q2, 0.0);
  for (int qd = 0; qd < 4; ++qd) {
    const int a = qd & 1, b = qd >> 1;
    for (int j2 = 0; j2 < q; ++j2)
      for (int j1 = 0; j1 < q; ++j1) {
        const int fr = qd * q2 + j1 + q * j2;
        for (int i2 = 0; i2 < q; ++i2)
          for (int i1 = 0; i1 < q; ++i1) {
            const int cr = i1 + q * i2;
            (*C2F)[(size_t)fr + (size_t)cr * 4 * q2] =
                c2f1[(size_t)(a * q + j1) * q + i1] * c2f1[(size_t)(b * q + j2) * q + i2];
            (*F2C)[(size_t)cr + (size_t)fr * q2] =
                f2c1[(size_t)i1 * 2 * q + a * q + j1] * f2c1[(size_t)i2 * 2 * q + b * q + j2];
          }
      }
  }
}

namespace {

struct CoarseEntry {
  Panel pn;
  bool fine_a, fine_b;
};

bool coarse_interface(const std::vector<Panel>& pa, const std::vector<Panel>& pb, Panel root,
                      std::vector<CoarseEntry>* out) {
  std::set<Panel> sa(pa.begin(), pa.end()), sb(pb.begin(), pb.end());
  bool ok = true;
  std::vector<Panel> stack = {root};
  // depth-first, children in Morton order: use explicit recursion for order
  struct Rec {
    const std::set<Panel>&sa, &sb;
    std::vector<CoarseEntry>* out;
    bool* ok;
    int max_level;
    void go(Panel p) {
      const bool ina = sa.count(p), inb = sb.count(p);
      if (ina || inb) {
        for (int side = 0; side < 2; ++side) {
          const bool here = side ? inb : ina;
          if (here) continue;
          const std::set<Panel>& s = side ? sb : sa;
          for (int qd = 0; qd < 4; ++qd) {
            Panel sub{p.level + 1, 2 * p.i1 + (qd & 1), 2 * p.i2 + (qd >> 1)};
            if (!s.count(sub)) *ok = false;
          }
        }
        out->push_back({p, !ina, !inb});
        return;
      }
      if (p.level >= max_level) { *ok = false; return; }
      for (int qd = 0; qd < 4; ++qd) go({p.level + 1, 2 * p.i1 + (qd & 1), 2 * p.i2 + (qd >> 1)});
    }
  };
  int maxl = 0;
  for (auto& p : pa) maxl = std::max(maxl, p.level);
  for (auto& p : pb) maxl = std::max(maxl, p.level);
  Rec r{sa, sb, out, &ok, maxl};
  r.go(root);
  (void)stack;
  return ok;
}

}  // namespace

bool build_atree(int p, int q, const double* lo, const double* hi, int64_t n_leaves, const uint64_t* morton,
                 const int8_t* level, ATree* out, const char** why) {
  ATree& t = *out;
  t = ATree();
  t.p = p;
  t.q = q;
  t.side = hi[0] - lo[0];
  for (int a = 0; a < 3; ++a) t.lo[a] = lo[a];
  if (n_leaves < 1 || !morton || !level) { *why = "empty leaf list"; return false; }
  std::map<Key, int> idx;
  t.nodes.push_back(ANode());  // root
  idx[{0, 0, 0, 0}] = 0;
  uint64_t prev = 0;
  t.leaf_node.resize(n_leaves);
  for (int64_t n = 0; n < n_leaves; ++n) {
    const int lv = level[n];
    if (lv < 0 || lv > 16) { *why = "leaf level out of range [0, 16]"; return false; }
    int64_t ix[3];
    morton_decode(morton[n], lv, ix);
    if (morton_encode(ix) != morton[n]) { *why = "Morton code has bits beyond its level"; return false; }
    const uint64_t key = dfs_key(lv, ix);
    if (n > 0 && key <= prev) { *why = "leaves are not in depth-first Morton order"; return false; }
    prev = key;
    t.max_level = std::max(t.max_level, lv);
    // create the chain of ancestors
    int parent = 0;
    for (int l = 1; l <= lv; ++l) {
      const int sh = lv - l;
      Key k{l, ix[0] >> sh, ix[1] >> sh, ix[2] >> sh};
      auto it = idx.find(k);
      int id;
      if (it == idx.end()) {
        ANode nd;
        nd.level = l;
        nd.ix[0] = k.x; nd.ix[1] = k.y; nd.ix[2] = k.z;
        id = (int)t.nodes.size();
        t.nodes.push_back(nd);
        idx[k] = id;
      } else {
        id = it->second;
      }
      if (t.nodes[parent].leaf >= 0) { *why = "a leaf contains another leaf"; return false; }
      const int c = (int)((k.x & 1) | ((k.y & 1) << 1) | ((k.z & 1) << 2));
      t.nodes[parent].child[c] = id;
      parent = id;
    }
    if (t.nodes[parent].leaf >= 0 || t.nodes[parent].child[0] >= 0) {
      *why = "duplicate or overlapping leaf";
      return false;
    }
    t.nodes[parent].leaf = (int)n;
    t.leaf_node[n] = parent;
  }
  // completeness: every merge node has 8 children
  for (auto& nd : t.nodes)
    if (nd.leaf < 0)
      for (int c = 0; c < 8; ++c)
        if (nd.child[c] < 0) { *why = "the leaves do not tile the cube"; return false; }
  // face panel lists, bottom-up by level
  std::vector<int> order(t.nodes.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return t.nodes[a].level > t.nodes[b].level; });
  const int q2 = q * q;
  for (int id : order) {
    ANode& nd = t.nodes[id];
    if (nd.leaf >= 0) {
      for (int f = 0; f < 6; ++f) {
        int tt[2];
        tang(kFaceAxis[f], tt);
        nd.faces[f] = {Panel{nd.level, nd.ix[tt[0]], nd.ix[tt[1]]}};
      }
    } else {
      for (int f = 0; f < 6; ++f) {
        int tt[2];
        tang(kFaceAxis[f], tt);
        nd.faces[f].clear();
        for (int qd = 0; qd < 4; ++qd) {
          int bits[3] = {0, 0, 0};
          bits[kFaceAxis[f]] = kFaceSide[f];
          bits[tt[0]] = qd & 1;
          bits[tt[1]] = qd >> 1;
          const int c = bits[0] | (bits[1] << 1) | (bits[2] << 2);
          const auto& cf = t.nodes[nd.child[c]].faces[f];
          nd.faces[f].insert(nd.faces[f].end(), cf.begin(), cf.end());
        }
      }
      t.merge_order.push_back(id);
    }
    int64_t np = 0;
    for (int f = 0; f < 6; ++f) np += (int64_t)nd.faces[f].size();
    nd.n_bdry = np * q2;
  }
  // merge plans
  t.plans.resize(t.merge_order.size());
  for (size_t mi = 0; mi < t.merge_order.size(); ++mi) {
    const int id = t.merge_order[mi];
    const ANode& nd = t.nodes[id];
    MergePlanA& pl = t.plans[mi];
    pl.node = id;
    // interfaces
    std::vector<CoarseEntry> iface[12];
    int var_off[12];
    int nv = 0;
    for (int axis = 0; axis < 3; ++axis) {
      int tt[2];
      tang(axis, tt);
      for (int c = 0; c < 8; ++c) {
        if ((c >> axis) & 1) continue;
        const int ch = c | (1 << axis);
        const ANode& A = t.nodes[nd.child[c]];
        const ANode& B = t.nodes[nd.child[ch]];
        const int sid = axis * 4 + ((c >> tt[0]) & 1) + 2 * ((c >> tt[1]) & 1);
        Panel root{A.level, A.ix[tt[0]], A.ix[tt[1]]};
        if (!coarse_interface(A.faces[2 * axis + 1], B.faces[2 * axis], root, &iface[sid])) {
          *why = "the tree is not 2:1 balanced across faces";
          return false;
        }
      }
    }
    for (int sid = 0; sid < 12; ++sid) {
      var_off[sid] = nv;
      nv += (int)iface[sid].size() * q2;
    }
    pl.n_int = nv;
    // parent boundary offsets per face panel
    std::map<Panel, int> poff[6];
    int o = 0;
    for (int f = 0; f < 6; ++f)
      for (const Panel& pn : nd.faces[f]) { poff[f][pn] = o; o += q2; }
    pl.n_ext = o;
    for (int c = 0; c < 8; ++c) {
      const ANode& K = t.nodes[nd.child[c]];
      ChildProj& cp = pl.ch[c];
      std::map<Panel, int> koff[6];
      int ko = 0;
      for (int f = 0; f < 6; ++f)
        for (const Panel& pn : K.faces[f]) { koff[f][pn] = ko; ko += q2; }
      cp.n = ko;
      cp.back_base.assign(ko, -1);
      cp.back_quad.assign(ko, -1);
      cp.back_t.assign(ko, -1);
      cp.back_copy.assign(ko, -1);
      int np = 0;
      for (int f = 0; f < 6; ++f) {
        const int axis = kFaceAxis[f], side = kFaceSide[f];
        int tt[2];
        tang(axis, tt);
        if (side == ((c >> axis) & 1)) {
          for (const Panel& pn : K.faces[f]) {
            const int src = koff[f][pn], dst = poff[f][pn];
            for (int u = 0; u < q2; ++u) {
              cp.kind.push_back(0);
              cp.u.push_back(u);
              cp.src.push_back({src + u, 0, 0, 0});
              cp.ext.push_back(dst + u);
              cp.var.push_back(-1);
              cp.back_copy[src + u] = np + u;
            }
            np += q2;
          }
          continue;
        }
        const bool low = side == 1;
        const int cc = low ? c : (c ^ (1 << axis));
        const int sid = axis * 4 + ((cc >> tt[0]) & 1) + 2 * ((cc >> tt[1]) & 1);
        for (size_t k = 0; k < iface[sid].size(); ++k) {
          const CoarseEntry& e = iface[sid][k];
          const bool fine = low ? e.fine_a : e.fine_b;
          const int vb = var_off[sid] + (int)k * q2;
          std::array<int, 4> srcs = {0, 0, 0, 0};
          if (!fine) {
            srcs[0] = koff[f][e.pn];
          } else {
            for (int qd = 0; qd < 4; ++qd) {
              Panel sub{e.pn.level + 1, 2 * e.pn.i1 + (qd & 1), 2 * e.pn.i2 + (qd >> 1)};
              srcs[qd] = koff[f][sub];
              for (int tq = 0; tq < q2; ++tq) {
                cp.back_base[srcs[qd] + tq] = np;
                cp.back_quad[srcs[qd] + tq] = qd;
                cp.back_t[srcs[qd] + tq] = tq;
              }
            }
          }
          for (int u = 0; u < q2; ++u) {
            cp.kind.push_back(fine ? 1 : 0);
            cp.u.push_back(u);
            if (fine) cp.src.push_back(srcs);
            else {
              cp.src.push_back({srcs[0] + u, 0, 0, 0});
              cp.back_copy[srcs[0] + u] = np + u;
            }
            cp.ext.push_back(-1);
            cp.var.push_back(vb + u);
          }
          np += q2;
        }
      }
      cp.np = np;
      for (int k = 0; k < np; ++k) {
        if (cp.ext[k] >= 0) { cp.b_arow.push_back(k); cp.b_crow.push_back(cp.ext[k]); }
        else { cp.b_acol.push_back(k); cp.b_brow.push_back(cp.var[k]); }
      }
    }
  }
  (void)why;
  return true;
}

void atree_leaf_coords(const ATree& t, const Spectral1D& s, double* out) {
  const int p = t.p, npts = p * p * p;
  for (size_t n = 0; n < t.leaf_node.size(); ++n) {
    const ANode& nd = t.nodes[t.leaf_node[n]];
    const double h = t.side / (double)((int64_t)1 << nd.level);
    for (int node = 0; node < npts; ++node) {
      const int c[3] = {node % p, (node / p) % p, node / (p * p)};
      for (int a = 0; a < 3; ++a)
        out[((size_t)n * npts + node) * 3 + a] = t.lo[a] + (nd.ix[a] + 0.5 * (s.xc[c[a]] + 1.0)) * h;
    }
  }
}

void atree_root_coords(const ATree& t, const Spectral1D& s, double* out) {
  const int q = t.q;
  const ANode& root = t.nodes[0];
  size_t o = 0;
  for (int f = 0; f < 6; ++f) {
    const int axis = kFaceAxis[f];
    int tt[2];
    tang(axis, tt);
    for (const Panel& pn : root.faces[f]) {
      const double h = t.side / (double)((int64_t)1 << pn.level);
      for (int b = 0; b < q; ++b)
        for (int a = 0; a < q; ++a) {
          out[o * 3 + axis] = t.lo[axis] + (kFaceSide[f] ? t.side : 0.0);
          out[o * 3 + tt[0]] = t.lo[tt[0]] + (pn.i1 + 0.5 * (s.xg[a] + 1.0)) * h;
          out[o * 3 + tt[1]] = t.lo[tt[1]] + (pn.i2 + 0.5 * (s.xg[b] + 1.0)) * h;
          ++o;
        }
    }
  }
}

}  // namespace hps
