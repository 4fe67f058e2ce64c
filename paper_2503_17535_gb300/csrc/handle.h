// Internal definition of the solver handle and small host helpers shared by
// the C ABI translation units.
#pragma once

#include <atomic>

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "devmem.h"
#include "adaptive.h"
#include "adaptive_kernels.cuh"
#include "hps.h"
#include "hps_kernels.cuh"
#include "linalg.h"
#include "plan.h"

namespace hps {

struct LevelDev {
  int nmerge = 0, nch = 0, n = 0, nbc = 0, n_ext = 0, n_int = 0;
  int *ext = nullptr, *var = nullptr, *eq = nullptr;
  int *barow = nullptr, *bacol = nullptr, *bbrow = nullptr, *bcrow = nullptr;
  // ItI interior blocks by parity: [2][nbc/2] interior points, own vars, eq rows
  int *odd_pts = nullptr, *odd_var = nullptr, *odd_eq = nullptr;
  int *even_pts = nullptr, *even_var = nullptr, *even_eq = nullptr;
  void* TP = nullptr;   // [nmerge][n_ext x (n_ext+1)]  parent [T | h]
  void* D = nullptr;    // [nmerge][n_int x n_int]
  void* W = nullptr;    // ItI: [nmerge][(n_int/2)^2] (LU of W)
  int* ipiv = nullptr;  // [nmerge][nlu]
  int* perm = nullptr;
  int* info = nullptr;  // [nmerge]
  void* X = nullptr;    // [nmerge][n_int x (n_ext+1)]  D^{-1} [C | h_int]
  int G = 1;
  LuWork luw;
  bool lazy = false;    // root only: X holds [C | h_int]; D^{-1} is applied per solve
  // adjoint B^H products of DtN levels, in two passes over the children of
  // even / odd popcount (children sharing an interface differ in one bit, so
  // no two products of one pass write the same interface rows): per pass a
  // device array of child [T | h] pointers and the four maps in pass order
  void* adj_ptrs[2] = {nullptr, nullptr};
  int* adj_maps[2] = {nullptr, nullptr};
  // solve workspace (nrhs columns)
  void *r = nullptr, *hp = nullptr, *x = nullptr, *gint = nullptr, *gchild = nullptr;
  bool top() const { return nmerge == 1; }
};

// Adaptive-tree storage: one merge of the nonuniform octree.
struct AChildDev {
  ProjDev pj;                 // projection descriptors (device arrays)
  int* ext = nullptr;         // per projected point
  int* var = nullptr;
  int *barow = nullptr, *bacol = nullptr, *bbrow = nullptr, *bcrow = nullptr;
  int ne_c = 0, ni_c = 0;     // exterior / interior projected points
  void* Tp = nullptr;         // np x (np + 1) projected [T | h]
};

// ItI leaves solved by elimination of the interior nodes (iti_leaf.cu): the
// real LU of L(I_i, I_i), W = L_ii^{-1} L(I_i, boundary), the complex LU of
// the boundary Schur complement S, and the shared real impedance-row blocks.
struct ItiElim {
  bool on = false;
  int ni = 0, no = 0;                      // interior nodes, boundary nodes (owner order)
  double *Goe = nullptr, *Goi = nullptr;   // shared: no x no, no x ni (real parts)
  double* LU = nullptr;                    // [leaf] ni x ni
  int *ipiv = nullptr, *perm = nullptr;
  double* W = nullptr;                     // [leaf] ni x no
  cplx* S = nullptr;                       // [leaf] no x no (LU)
  int *ipivS = nullptr, *permS = nullptr;
  LuWork luw, luwS;
  int G = 1, GS = 1;
  int cap = 0;                             // columns the workspace holds
  double *z = nullptr, *z2 = nullptr, *t = nullptr;
  cplx *q = nullptr, *q2 = nullptr;
};

// Merges of one tree level with the same interface sizes: their dense
// factorisations and solves run as one batched call (pointer arrays).
struct AGroup {
  int level = 0, n_int = 0, n_ext = 0, G = 1;
  std::vector<int> members;      // indices into hps_handle::am
  LuWork luw;
  int *ipiv = nullptr, *perm = nullptr, *info = nullptr;  // [members][n_int], [members]
  double **dD = nullptr, **dX = nullptr, **dR = nullptr;  // build operands
  double **dTP = nullptr;                                 // parents' [T | h]
  double **dr = nullptr, **dx = nullptr, **dhp = nullptr; // solve workspace
  // per child position: when every member's child has the same projected
  // sizes, one batched B X product over the group (maps concatenated,
  // period = members), else one product per member
  struct ChildBatch {
    bool ok = false;
    int ne_c = 0, ni_c = 0, np = 0;
    int *barow = nullptr, *bacol = nullptr, *bbrow = nullptr, *bcrow = nullptr;
    double** dTp = nullptr;
  } cb[8];
};

// The solve passes of one level of an adaptive tree as grouped launches:
// device task tables (built with the solve workspace) and their sizes.
struct ASolveLevel {
  std::vector<int> merges;            // indices into am
  ZeroTask<double>* zr = nullptr;     // up: zero r of every merge
  ProjTask<double>* pr = nullptr;     // up: each child's h projected
  ChildTask<double>* gh = nullptr;    // up: projected h into r and hp
  GintTask<double>* gi = nullptr;     // down: gint of the non-lazy merges
  ChildTask<double>* dc = nullptr;    // down: each child's projected data
  ProjTask<double>* un = nullptr;     // down: unprojected onto the child
  int nzr = 0, npr = 0, ngh = 0, ngi = 0, ndc = 0, nun = 0;
  int64_t tzr = 0, tpr = 0, tgh = 0, tgi = 0, tdc = 0, tun = 0;
};

struct AMergeDev {
  int node = -1, n_ext = 0, n_int = 0;
  AChildDev ch[8];
  void *D = nullptr, *X = nullptr, *TP = nullptr;
  int *ipiv = nullptr, *perm = nullptr, *info = nullptr;
  int G = 1;
  LuWork luw;
  bool lazy = false;  // root only: X holds [C | h_int]; D^{-1} is applied per solve
  // solve workspace (nrhs columns)
  void *r = nullptr, *x = nullptr, *hp = nullptr, *gint = nullptr, *g = nullptr;
};

}  // namespace hps

using hps::ATree;
using hps::ASolveLevel;
using hps::ItiElim;
using hps::cplx;
using hps::DtnLeafRef;
using hps::ItiLeafRef;
using hps::LeafConsts;
using hps::LevelDev;
using hps::LuWork;
using hps::Prof;
using hps::Spectral1D;

struct hps_handle {
  int dim = 0, kind = 0, p = 0, q = 0, L = 0;
  bool iti = false;
  int64_t nl = 0, npts = 0, nroot = 0;
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, eta = 0.0, hlen = 0.0, s = 0.0;
  hps_options opts{};
  Spectral1D spec;
  DtnLeafRef dref;
  ItiLeafRef iref;
  LeafConsts lc{};
  int nlu_leaf = 0, xrows_leaf = 0, nb = 0;
  // device constants
  double *dD = nullptr, *dDD = nullptr, *dP = nullptr, *dQi = nullptr, *dQP = nullptr, *dsgn = nullptr;
  int *dIi = nullptr, *dprow = nullptr, *diidx = nullptr, *downn = nullptr, *downa = nullptr;
  cplx* dQH = nullptr;
  // leaf storage
  void* leafA = nullptr;  // LU of L_ii (DtN) or B (ItI)
  int *leaf_ipiv = nullptr, *leaf_perm = nullptr, *leaf_info = nullptr;
  void* leafX = nullptr;  // DtN: X = L_ii^{-1}[L_ie P | -f_i]; ItI: [Y | v]
  void* leafTH = nullptr; // [T | h]
  LuWork leaf_luw;
  int leaf_G = 1;
  std::vector<LevelDev> lev;
  unsigned* dev_err = nullptr;
  void* scratch = nullptr;  // build-time R / RHS buffer
  std::vector<void*> allocs;
  int64_t bytes = 0;
  Prof prof;
  hps::TcWorkspace tcw;           // digit slices of tensor-core products (build only)
  int64_t err_node = -1;
  int num_sms = 0;
  int device = -1;               // CUDA device the handle was built on
  // Subtree recomputation (hps_options.recompute_budget_mb; paper Section
  // 4.1, Algorithm "our_recomputation").  A composite handle (recompute)
  // keeps only `top` -- a handle whose leaves are the roots of the complete
  // subtrees of depth sub_depth (ext_depth > 0 there, their T and h in
  // leafTH) -- and device copies of the coefficients and the build-time
  // source; every solve rebuilds each subtree on its way down.
  int ext_depth = 0;             // leaves of this handle: roots of subtrees of this depth
  int n0 = 0;                    // Gauss points per side (2D) / face panel (3D) at the first merge; 0: q (q^2)
  bool ext_newf = false;         // solve: the leaves' h for the new sources are already in ws_hleaf
  bool recompute = false;
  hps_handle* top = nullptr;
  int sub_depth = 0;
  const double* rc_coef[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // a, b[0..2], c
  void* rc_f = nullptr;          // build-time source (null: f = 0)
  void* rc_u = nullptr;          // one subtree's solutions for nrhs right-hand sides
  int64_t rc_u_elems = 0;
  // captured solves (hps_options.graph_solve): key -> executable graph
  struct GraphEntry {
    int nrhs = 0;
    const void *g = nullptr, *f = nullptr;
    void* u = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool warm = false;  // seen once (workspace allocated), not captured yet
  };
  std::vector<GraphEntry> graphs;
  bool capturing = false;
  hps::ItiElim ie;               // ItI leaves by interior elimination (when on)
  hps::TrsvWork trsv;            // flag-ordered solves with a lazy root's factors
  int* trsv_err_host = nullptr;  // host-mapped error word of trsv (cudaHostAlloc)
  cudaStream_t last = nullptr;
  // Completion of the handle's latest work, whatever stream it ran on: each
  // call that enqueues work on the handle first orders its stream after this
  // event and records it again at its end, so calls made on different
  // streams never overlap on the handle's buffers, and hps_free waits for
  // exactly the handle's own work.
  cudaEvent_t done = nullptr;
  bool done_recorded = false;
  // solve workspace
  int ws_nrhs = 0;
  // adaptive trees
  bool adaptive = false;
  ATree at;
  std::vector<hps::AMergeDev> am;
  std::vector<hps::AGroup> ag;   // batched groups, deepest level first
  std::vector<hps::ASolveLevel> alev;  // solve passes per level, deepest first
  std::vector<int> node_merge;   // tree node -> index in am, or -1
  double *dC2F = nullptr, *dF2C = nullptr, *dsleaf = nullptr;
  void* aproj_tmp = nullptr;     // projection temporaries (build)
  void* ws_vtmp = nullptr;       // projected-vector temporary (solve)
  int max_np = 0;
  int64_t ws_bytes = 0;
  std::vector<void*> ws_allocs;
  void *ws_xf = nullptr, *ws_hleaf = nullptr, *ws_gleaf = nullptr, *ws_g = nullptr, *ws_f = nullptr,
       *ws_u = nullptr, *ws_rhs = nullptr;
};

namespace hps {

#define HPS_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      return HPS_ERR_CUDA;                              \
    }                                                   \
  } while (0)

// Solve workspace for nrhs columns (uniform trees); defined with the solve.
hps_status ensure_solve_ws(hps_handle* h, int nrhs);
// Adjoint solve and coefficient gradients (uniform trees), hps_adjoint.cu.
hps_status adjoint_solve(hps_handle* h, int nrhs, const void* ubar, void* gbar, void* fbar, cudaStream_t st);
hps_status coeff_gradient(hps_handle* h, int nrhs, const void* u, const void* fbar, double* ga, double* gb,
                          double* gc, cudaStream_t st);

// ItI interior elimination (iti_leaf.cu): whether to use it for these
// coefficients (hps_options.iti_leaf, or the resonance check), the setup
// (factorisations), X = B^{-1} R and Rbar = B^{-H} Xbar per leaf (R in B's
// rows order, X in node order; p^2 x m per leaf).
bool iti_elim_safe(hps_handle* h, const Coeffs& co, cudaStream_t st, hps_status* err);
hps_status iti_elim_setup(hps_handle* h, const Coeffs& co, cudaStream_t st, Prof* pf);
hps_status iti_elim_apply(hps_handle* h, const cplx* R, cplx* X, int m, cudaStream_t st, Prof* pf);
hps_status iti_elim_apply_h(hps_handle* h, const cplx* Xb, cplx* Rb, int m, cudaStream_t st, Prof* pf);

#define HPS_TRY(call)                                   \
  do {                                                  \
    hps_status s_ = (call);                             \
    if (s_ != HPS_OK) return s_;                        \
  } while (0)

// Host-side fault injection for tests (hps_debug_fail_alloc): a countdown
// of handle allocations; the allocation that takes it from 1 to 0 fails as
// if cudaMalloc had run out of memory.  Also counts all handle allocations.
std::atomic<int64_t>& alloc_fail_countdown();
std::atomic<int64_t>& alloc_counter();

inline void* dalloc(hps_handle* h, size_t bytes, std::vector<void*>* list = nullptr) {
  if (bytes == 0) bytes = 16;
  alloc_counter().fetch_add(1);
  {
    std::atomic<int64_t>& c = alloc_fail_countdown();
    int64_t v = c.load();
    while (v > 0 && !c.compare_exchange_weak(v, v - 1)) {}
    if (v == 1) return nullptr;
  }
  void* p = nullptr;
  if (dev_malloc(&p, bytes, h->last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  (list ? *list : h->allocs).push_back(p);
  h->bytes += (int64_t)bytes;
  return p;
}

template <typename V>
V* upload(hps_handle* h, const std::vector<V>& v, cudaStream_t st) {
  V* d = (V*)dalloc(h, v.size() * sizeof(V));
  if (!d) return nullptr;
  if (cudaMemcpyAsync(d, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return nullptr;
  return d;
}

inline bool is_device_ptr(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T> struct Kind;
template <> struct Kind<double> { static constexpr bool iti = false; };
template <> struct Kind<cplx> { static constexpr bool iti = true; };

}  // namespace hps
