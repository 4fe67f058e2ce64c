// Adaptive-tree entry points used by the C ABI (hps_capi.cu).
#pragma once

#include "handle.h"

namespace hps {

// Validate an hps_tree with uniform_depth == -1 and build the octree plan.
hps_status adaptive_tree_from_abi(const hps_tree* t, int p, int q, ATree* out);

hps_status adaptive_build(hps_handle* h, const hps_tree* tree, const hps_coeffs* cf, const void* f,
                          cudaStream_t st);

hps_status adaptive_solve(hps_handle* h, int nrhs, const void* g, const void* f, void* u, cudaStream_t st);

hps_status adaptive_refine(const double* lo, const double* hi, int p, double eps, int min_depth, int max_depth,
                           int n_fn, const hps_eval_fn* fns, void* const* ctxs, int64_t capacity,
                           int64_t* n_leaves, uint64_t* morton, int8_t* level, cudaStream_t st);

}  // namespace hps
