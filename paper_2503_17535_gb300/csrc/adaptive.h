// Adaptive octrees (Section 4.2): tree validation from a leaf list, node face
// panel lists, the per-merge plan of the nonuniform merge (coarse interface
// panels, 4-to-1 projections, scatter maps), 2:1 balancing and the 4-to-1
// panel projection operators.  Host code only.
#pragma once

#include <array>
#include <cstdint>
#include <map>
#include <vector>

#include "plan.h"

namespace hps {

struct Panel {
  int level;
  int64_t i1, i2;
  bool operator<(const Panel& o) const {
    if (level != o.level) return level < o.level;
    if (i1 != o.i1) return i1 < o.i1;
    return i2 < o.i2;
  }
  bool operator==(const Panel& o) const { return level == o.level && i1 == o.i1 && i2 == o.i2; }
};

struct ANode {
  int level = 0;
  int64_t ix[3] = {0, 0, 0};
  int leaf = -1;                  // leaf number, or -1 for a merge node
  int child[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
  std::vector<Panel> faces[6];    // quadtree order
  int64_t n_bdry = 0;
};

// Projected representation of one child inside one merge: the child's
// boundary with every fine interface group replaced by its coarse panel.
struct ChildProj {
  int n = 0;        // child boundary points
  int np = 0;       // projected points
  // per projected point: kind 0 = copy of child point src[0], 1 = coarse
  // point u of a group whose 4 fine panels start at src[0..3]
  std::vector<int> kind, u;
  std::vector<std::array<int, 4>> src;
  // per child point: projected panel start of its group and the fine quadrant
  // (-1 for copied points) and the copy source (projected index) otherwise
  std::vector<int> back_base, back_quad, back_t, back_copy;
  std::vector<int> ext, var;                  // per projected point
  std::vector<int> b_arow, b_crow, b_acol, b_brow;  // exterior / interior lists
};

struct MergePlanA {
  int node = -1;
  int n_ext = 0, n_int = 0;
  ChildProj ch[8];
};

struct ATree {
  int p = 0, q = 0;
  double lo[3] = {0, 0, 0}, side = 0.0;
  std::vector<ANode> nodes;        // nodes[0] = root
  std::vector<int> leaf_node;      // leaf number -> node index
  std::vector<int> merge_order;    // merge nodes, deepest level first
  std::vector<MergePlanA> plans;   // aligned with merge_order
  int max_level = 0;
};

// Build from leaves given as (level, Morton code of the integer coordinates
// at that level, x in the lowest bit).  The leaves must tile the cube, be in
// depth-first Morton order and be 2:1 balanced across faces.  Returns false
// (with a reason) otherwise.
bool build_atree(int p, int q, const double* lo, const double* hi, int64_t n_leaves,
                 const uint64_t* morton, const int8_t* level, ATree* out, const char** why);

// 4-to-1 projections on one face panel (column-major):
//   C2F: 4q^2 x q^2  coarse data -> the 4 fine panels (Morton over t1, t2)
//   F2C: q^2 x 4q^2  L2 projection of fine data onto the coarse panel
void panel_projections(const Spectral1D& s, std::vector<double>* C2F, std::vector<double>* F2C);

// Coordinates: leaf Chebyshev nodes and root boundary Gauss points.
void atree_leaf_coords(const ATree& t, const Spectral1D& s, double* out);
void atree_root_coords(const ATree& t, const Spectral1D& s, double* out);

// Level-by-level refinement helpers.
uint64_t morton_encode(const int64_t* ix);
void morton_decode(uint64_t code, int level, int64_t* ix);
// Split leaves with a face neighbour two or more levels finer until none is left.
void balance_leaves(std::vector<std::pair<int, std::array<int64_t, 3>>>* leaves);
void sort_leaves(std::vector<std::pair<int, std::array<int64_t, 3>>>* leaves);

}  // namespace hps
