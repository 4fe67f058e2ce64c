// Host precompute: spectral nodes, differentiation and interpolation
// matrices, reference leaf operators and merge index maps.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace hps {

namespace {

// Legendre P_q and its derivative at x by the three-term recurrence.
void legendre(int q, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (q == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= q; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = q * (x * p1 - p0) / (x * x - 1.0);
}

// Gauss--Legendre nodes: Newton's method on P_q from the Chebyshev-like
// initial guesses cos(pi (i + 3/4) / (q + 1/2)).
std::vector<double> gauss_nodes(int q) {
  std::vector<double> x(q);
  const double pi = std::acos(-1.0);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(pi * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(q, z, &P, &dP);
      double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  std::sort(x.begin(), x.end());
  return x;
}

std::vector<double> bary_w(const std::vector<double>& x) {
  const int n = (int)x.size();
  std::vector<double> w(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) w[j] *= (x[j] - x[k]);
  double mx = 0.0;
  for (int j = 0; j < n; ++j) { w[j] = 1.0 / w[j]; mx = std::max(mx, std::fabs(w[j])); }
  for (auto& v : w) v /= mx;
  return w;
}

// Barycentric interpolation (second form) from nodes s to points t, row-major.
std::vector<double> interp(const std::vector<double>& s, const std::vector<double>& t) {
  const int m = (int)t.size(), n = (int)s.size();
  std::vector<double> w = bary_w(s), M((size_t)m * n, 0.0);
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

inline int node_index(int dim, int p, const int* c) {
  return dim == 2 ? c[0] + p * c[1] : c[0] + p * (c[1] + p * c[2]);
}
inline void node_coords(int dim, int p, int idx, int* c) {
  c[0] = idx % p;
  c[1] = (idx / p) % p;
  if (dim == 3) c[2] = idx / (p * p);
}

// Boundary faces of a leaf in canonical order: 2D S, E, N, W; 3D -x..+z.
struct Face { int axis, side; };
std::vector<Face> faces_of(int dim) {
  if (dim == 2) return {{1, 0}, {0, 1}, {1, 1}, {0, 0}};
  return {{0, 0}, {0, 1}, {1, 0}, {1, 1}, {2, 0}, {2, 1}};
}
// Tangential axes of a face (ascending).
void tangential(int dim, int axis, int* t) {
  int k = 0;
  for (int a = 0; a < dim; ++a)
    if (a != axis) t[k++] = a;
}

}  // namespace

Spectral1D make_spectral(int p, int q) {
  Spectral1D s;
  s.p = p;
  s.q = q;
  const double pi = std::acos(-1.0);
  s.xc.resize(p);
  for (int j = 0; j < p; ++j) s.xc[j] = -std::cos(pi * j / (p - 1));
  s.xg = gauss_nodes(q);
  // Chebyshev--Lobatto barycentric weights (-1)^j delta_j, delta = 1/2 at the ends
  std::vector<double> w(p);
  for (int j = 0; j < p; ++j) w[j] = ((j % 2) ? -1.0 : 1.0) * ((j == 0 || j == p - 1) ? 0.5 : 1.0);
  s.D.assign((size_t)p * p, 0.0);
  for (int i = 0; i < p; ++i) {
    double diag = 0.0;
    for (int j = 0; j < p; ++j) {
      if (i == j) continue;
      double v = (w[j] / w[i]) / (s.xc[i] - s.xc[j]);
      s.D[(size_t)i * p + j] = v;
      diag -= v;
    }
    s.D[(size_t)i * p + i] = diag;
  }
  s.DD.assign((size_t)p * p, 0.0);
  for (int i = 0; i < p; ++i)
    for (int k = 0; k < p; ++k)
      for (int j = 0; j < p; ++j) s.DD[(size_t)i * p + j] += s.D[(size_t)i * p + k] * s.D[(size_t)k * p + j];
  s.G2C = interp(s.xg, s.xc);
  s.C2G = interp(s.xc, s.xg);
  return s;
}

DtnLeafRef make_dtn_leaf(const Spectral1D& s, int dim) {
  DtnLeafRef r;
  const int p = s.p, q = s.q;
  r.dim = dim; r.p = p; r.q = q;
  r.npts = dim == 2 ? p * p : p * p * p;
  const int fq = dim == 2 ? q : q * q;       // Gauss points per face
  const int fp = dim == 2 ? p : p * p;       // Chebyshev points per face
  const auto faces = faces_of(dim);
  r.nb = (int)faces.size() * fq;
  r.prow.assign(r.npts, -1);
  for (int idx = 0; idx < r.npts; ++idx) {
    int c[3] = {0, 0, 0};
    node_coords(dim, p, idx, c);
    bool inner = true;
    for (int a = 0; a < dim; ++a) inner = inner && c[a] > 0 && c[a] < p - 1;
    if (inner) r.Ii.push_back(idx);
    else { r.prow[idx] = (int)r.Ie.size(); r.Ie.push_back(idx); }
  }
  r.ni = (int)r.Ii.size();
  r.ne = (int)r.Ie.size();
  // face node lists (tensor order over the tangential axes, lower axis fastest)
  std::vector<std::vector<int>> fnodes(faces.size());
  for (size_t f = 0; f < faces.size(); ++f) {
    int t[2] = {0, 0};
    tangential(dim, faces[f].axis, t);
    for (int k = 0; k < fp; ++k) {
      int c[3] = {0, 0, 0};
      c[faces[f].axis] = faces[f].side ? p - 1 : 0;
      c[t[0]] = k % p;
      if (dim == 3) c[t[1]] = k / p;
      fnodes[f].push_back(node_index(dim, p, c));
    }
  }
  // P: average of the face interpolants over the faces that contain the node
  r.P.assign((size_t)r.ne * r.nb, 0.0);
  for (int e = 0; e < r.ne; ++e) {
    const int node = r.Ie[e];
    std::vector<std::pair<int, int>> hits;
    for (size_t f = 0; f < faces.size(); ++f)
      for (int k = 0; k < fp; ++k)
        if (fnodes[f][k] == node) hits.push_back({(int)f, k});
    const double wgt = 1.0 / hits.size();
    for (auto& hk : hits) {
      const int f = hk.first, k = hk.second;
      if (dim == 2) {
        for (int j = 0; j < q; ++j)
          r.P[(size_t)e + (size_t)(f * fq + j) * r.ne] += wgt * s.G2C[(size_t)k * q + j];
      } else {
        const int i1 = k % p, i2 = k / p;
        for (int j2 = 0; j2 < q; ++j2)
          for (int j1 = 0; j1 < q; ++j1)
            r.P[(size_t)e + (size_t)(f * fq + j1 + q * j2) * r.ne] +=
                wgt * s.G2C[(size_t)i1 * q + j1] * s.G2C[(size_t)i2 * q + j2];
      }
    }
  }
  // Q (scale 1): for face f, rows f*fq..: interp(C->G) applied to the outward
  // normal derivative at the face's Chebyshev nodes.
  std::vector<double> Q((size_t)r.nb * r.npts, 0.0);  // row-major nb x npts
  for (size_t f = 0; f < faces.size(); ++f) {
    const int axis = faces[f].axis;
    const double sgn = faces[f].side ? 1.0 : -1.0;
    for (int k = 0; k < fp; ++k) {
      const int node = fnodes[f][k];
      int c[3] = {0, 0, 0};
      node_coords(dim, p, node, c);
      // normal derivative row at node: sgn * D[c_axis][m] along axis
      for (int m = 0; m < p; ++m) {
        int c2[3] = {c[0], c[1], c[2]};
        c2[axis] = m;
        const int col = node_index(dim, p, c2);
        const double dval = sgn * s.D[(size_t)c[axis] * p + m];
        if (dval == 0.0) continue;
        if (dim == 2) {
          for (int j = 0; j < q; ++j)
            Q[(size_t)(f * fq + j) * r.npts + col] += s.C2G[(size_t)j * p + k] * dval;
        } else {
          const int i1 = k % p, i2 = k / p;
          for (int j2 = 0; j2 < q; ++j2)
            for (int j1 = 0; j1 < q; ++j1)
              Q[(size_t)(f * fq + j1 + q * j2) * r.npts + col] +=
                  s.C2G[(size_t)j1 * p + i1] * s.C2G[(size_t)j2 * p + i2] * dval;
        }
      }
    }
  }
  r.Qi.assign((size_t)r.nb * r.ni, 0.0);
  for (int i = 0; i < r.nb; ++i)
    for (int c = 0; c < r.ni; ++c) r.Qi[(size_t)i + (size_t)c * r.nb] = Q[(size_t)i * r.npts + r.Ii[c]];
  r.QP.assign((size_t)r.nb * r.nb, 0.0);
  for (int i = 0; i < r.nb; ++i)
    for (int e = 0; e < r.ne; ++e) {
      const double qv = Q[(size_t)i * r.npts + r.Ie[e]];
      if (qv == 0.0) continue;
      for (int j = 0; j < r.nb; ++j) r.QP[(size_t)i + (size_t)j * r.nb] += qv * r.P[(size_t)e + (size_t)j * r.ne];
    }
  return r;
}

ItiLeafRef make_iti_leaf(const Spectral1D& s) {
  ItiLeafRef r;
  const int p = s.p, q = s.q;
  r.p = p; r.q = q; r.npts = p * p; r.nb = 4 * q; r.nown = 4 * (p - 1);
  // counterclockwise ownership: S x = 0..p-2, E y = 0..p-2, N x = 1..p-1, W y = 1..p-1
  const auto faces = faces_of(2);
  r.P.assign((size_t)r.nown * r.nb, 0.0);
  int row = 0;
  for (int f = 0; f < 4; ++f) {
    const int axis = faces[f].axis;
    const int lo = (f < 2) ? 0 : 1, hi = (f < 2) ? p - 2 : p - 1;
    for (int k = lo; k <= hi; ++k) {
      int c[3] = {0, 0, 0};
      c[axis] = faces[f].side ? p - 1 : 0;
      c[1 - axis] = k;
      r.own_node.push_back(node_index(2, p, c));
      r.own_axis.push_back(axis);
      r.own_sgn.push_back(faces[f].side ? 1.0 : -1.0);
      for (int j = 0; j < q; ++j) r.P[(size_t)row + (size_t)(f * q + j) * r.nown] = s.G2C[(size_t)k * q + j];
      ++row;
    }
  }
  for (int iy = 1; iy < p - 1; ++iy)
    for (int ix = 1; ix < p - 1; ++ix) r.Ii.push_back(ix + p * iy);
  return r;
}

std::vector<std::complex<double>> make_iti_QH(const Spectral1D& s, double hlen, double eta) {
  const int p = s.p, q = s.q, npts = p * p, nb = 4 * q;
  const double sc = 2.0 / hlen;
  std::vector<std::complex<double>> QH((size_t)nb * npts, 0.0);
  const auto faces = faces_of(2);
  for (int f = 0; f < 4; ++f) {
    const int axis = faces[f].axis;
    const double sgn = faces[f].side ? 1.0 : -1.0;
    for (int k = 0; k < p; ++k) {
      int c[3] = {0, 0, 0};
      c[axis] = faces[f].side ? p - 1 : 0;
      c[1 - axis] = k;
      const int node = node_index(2, p, c);
      // H row for this side point: sgn * sc * D_axis - i eta e_node
      for (int j = 0; j < q; ++j) {
        const double w = s.C2G[(size_t)j * p + k];
        const size_t rowi = (size_t)(f * q + j);
        for (int m = 0; m < p; ++m) {
          int c2[3] = {c[0], c[1], 0};
          c2[axis] = m;
          const int col = node_index(2, p, c2);
          QH[rowi + (size_t)col * nb] += w * sgn * sc * s.D[(size_t)c[axis] * p + m];
        }
        QH[rowi + (size_t)node * nb] += std::complex<double>(0.0, -eta * w);
      }
    }
  }
  return QH;
}

MergeMaps make_merge_maps(int dim, int n, bool iti) {
  MergeMaps m;
  m.dim = dim; m.n = n; m.iti = iti;
  m.nch = dim == 2 ? 4 : 8;
  const auto faces = faces_of(dim);
  const int nf = (int)faces.size();
  m.nbc = nf * n;
  const int per_face_parent = dim == 2 ? 2 * n : 4 * n;
  m.n_ext = nf * per_face_parent;
  const int n_if = dim == 2 ? 4 : 12;         // interfaces
  m.n_int = iti ? 2 * n_if * n : n_if * n;
  m.ext.assign((size_t)m.nch * m.nbc, -1);
  m.var.assign((size_t)m.nch * m.nbc, -1);
  m.eq.assign((size_t)m.nch * m.nbc, -1);
  const int half = n_if * n;
  for (int k = 0; k < m.nch; ++k) {
    int cb[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
    const bool even = ((cb[0] + cb[1]) % 2) == 0;
    for (int f = 0; f < nf; ++f) {
      const int axis = faces[f].axis, side = faces[f].side;
      int t[2] = {0, 0};
      tangential(dim, axis, t);
      for (int i = 0; i < n; ++i) {
        const size_t slot = (size_t)k * m.nbc + f * n + i;
        if (side == cb[axis]) {
          const int quad = dim == 2 ? cb[t[0]] : cb[t[0]] + 2 * cb[t[1]];
          m.ext[slot] = f * per_face_parent + quad * n + i;
        } else {
          const int id = dim == 2 ? axis * 2 + cb[t[0]] : axis * 4 + cb[t[0]] + 2 * cb[t[1]];
          if (!iti) {
            m.var[slot] = id * n + i;
            m.eq[slot] = id * n + i;
          } else {
            const int own = (even ? 0 : half) + id * n + i;
            const int oth = (even ? half : 0) + id * n + i;
            m.var[slot] = own;
            m.eq[slot] = oth;
          }
        }
      }
    }
    for (int i = 0; i < m.nbc; ++i) {
      const size_t slot = (size_t)k * m.nbc + i;
      if (m.ext[slot] >= 0) { m.b_arow.push_back(i); m.b_crow.push_back(m.ext[slot]); }
      else { m.b_acol.push_back(i); m.b_brow.push_back(m.var[slot]); m.i_eq.push_back(m.eq[slot]); }
    }
  }
  if ((int)m.b_arow.size() != m.nch * m.nbc / 2) throw std::runtime_error("merge map size");
  return m;
}

void leaf_node_coords(int dim, const double* lo, const double* hi, int L, const Spectral1D& s,
                      double* out) {
  const int p = s.p;
  const int64_t n1 = (int64_t)1 << L;
  const int64_t nl = dim == 2 ? n1 * n1 : n1 * n1 * n1;
  const int npts = dim == 2 ? p * p : p * p * p;
  double h[3];
  for (int a = 0; a < dim; ++a) h[a] = (hi[a] - lo[a]) / n1;
  for (int64_t m = 0; m < nl; ++m) {
    int64_t idx[3] = {0, 0, 0};
    for (int lev = 0; lev < L; ++lev) {
      const int c = (int)((m >> (dim * (L - 1 - lev))) & ((1 << dim) - 1));
      for (int a = 0; a < dim; ++a) idx[a] = idx[a] * 2 + ((c >> a) & 1);
    }
    for (int node = 0; node < npts; ++node) {
      int c[3] = {0, 0, 0};
      node_coords(dim, p, node, c);
      for (int a = 0; a < dim; ++a)
        out[((size_t)m * npts + node) * dim + a] = lo[a] + (idx[a] + 0.5 * (s.xc[c[a]] + 1.0)) * h[a];
    }
  }
}

void root_boundary_coords(int dim, const double* lo, const double* hi, int L, const Spectral1D& s,
                          double* out) {
  const int q = s.q;
  const int64_t n1 = (int64_t)1 << L;
  double h[3];
  for (int a = 0; a < dim; ++a) h[a] = (hi[a] - lo[a]) / n1;
  const auto faces = faces_of(dim);
  size_t o = 0;
  for (const auto& fc : faces) {
    int t[2] = {0, 0};
    tangential(dim, fc.axis, t);
    if (dim == 2) {
      for (int64_t i = 0; i < n1; ++i)
        for (int j = 0; j < q; ++j) {
          out[o * 2 + fc.axis] = fc.side ? hi[fc.axis] : lo[fc.axis];
          out[o * 2 + t[0]] = lo[t[0]] + (i + 0.5 * (s.xg[j] + 1.0)) * h[t[0]];
          ++o;
        }
    } else {
      const int64_t npan = n1 * n1;
      for (int64_t mm = 0; mm < npan; ++mm) {
        int64_t i1 = 0, i2 = 0;
        for (int lev = 0; lev < L; ++lev) {
          const int c = (int)((mm >> (2 * (L - 1 - lev))) & 3);
          i1 = i1 * 2 + (c & 1);
          i2 = i2 * 2 + (c >> 1);
        }
        for (int b = 0; b < q; ++b)
          for (int a = 0; a < q; ++a) {
            out[o * 3 + fc.axis] = fc.side ? hi[fc.axis] : lo[fc.axis];
            out[o * 3 + t[0]] = lo[t[0]] + (i1 + 0.5 * (s.xg[a] + 1.0)) * h[t[0]];
            out[o * 3 + t[1]] = lo[t[1]] + (i2 + 0.5 * (s.xg[b] + 1.0)) * h[t[1]];
            ++o;
          }
      }
    }
  }
}

}  // namespace hps
