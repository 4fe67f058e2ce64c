/*
 * hps.h -- C ABI of the GB300 (sm_103a) HPS fast direct solver.
 *
 * Hierarchical Poincare--Steklov solver for L u = a(x) Lap u + b(x).grad u
 * + c(x) u = f on a square or cube with Dirichlet data (DtN variant) or
 * incoming impedance data u_n + i eta u (ItI variant), after arXiv 2503.17535:
 *   leaf stage     Section 3.2, Algorithms "2D DtN local solve" (App. A.1),
 *                  "2D ItI local solve" (App. B.1), 3D DtN (App. C.1);
 *   merge stage    Section 3.3, Eqs. "merge linear system", "merge outputs
 *                  1-2", block formulas of Apps. A.2, B.2 (with the W route of
 *                  Eq. "ItI D inverse") and C.2;
 *   downward pass  Section 3.4, Algorithm "down pass".
 *
 * Conventions shared by every entry point:
 *   - Leaves of a uniform tree of depth L: 2^(dL), numbered depth first with
 *     children in Morton order c = cx + 2 cy (+ 4 cz) (leaf numbers are Morton
 *     codes, coarsest level in the most significant bits).
 *   - Per-leaf arrays ("leaf-major"): [n_leaves][p^d], nodes of one leaf in
 *     tensor order, x fastest: (ix, iy, iz) -> ix + p iy + p^2 iz, where the p
 *     Chebyshev--Lobatto points of each axis are ascending.
 *   - Root boundary data g: the root's Gauss--Legendre points (q = p - 2 per
 *     leaf side) ordered by sides S, E, N, W (2D: y = lo, x = hi, y = hi,
 *     x = lo; each side by increasing coordinate) or by faces -x, +x, -y, +y,
 *     -z, +z (3D: each face is the quadtree of its leaf panels in Morton order
 *     over its two tangential axes, lower axis first; q^2 points per panel in
 *     tensor order, lower tangential axis fastest).  hps_nodes() returns the
 *     coordinates in exactly these orders.
 *   - DtN: g = Dirichlet values u.  ItI: g = u_n + i eta u with the outward
 *     normal (Section 2).  Real data is double; complex data is interleaved
 *     (re, im) double pairs (C99 double complex / std::complex<double>).
 *
 * Memory: every pointer argument may be device memory (cudaMalloc /
 * cudaMallocManaged) or host memory.  Host buffers are staged through the
 * handle's own device buffers on the given stream (the call then returns
 * after the copy back has completed).  The caller owns every buffer it passes;
 * the library copies what it keeps.  The handle owns all factor storage.
 *
 * Streams: work is enqueued on the stream passed in (NULL = legacy default
 * stream).  hps_build and hps_solve are asynchronous with respect to the host
 * for device buffers, except that hps_build synchronises the stream once at
 * its end to read the pivot status.  Calls on one handle made on different
 * streams are ordered on the device: each call's stream first waits for the
 * handle's previous work (an event the handle records), so they never
 * overlap on the handle's buffers (not while the caller captures the stream
 * into a graph, where the caller's graph orders the work).  A handle must
 * not be used from two host threads at the same time.
 *
 * Device memory of handles and their workspaces comes from a stream-ordered
 * pool per device (cudaMallocFromPoolAsync / cudaFreeAsync, release
 * threshold 0): building, growing a workspace or freeing a handle never
 * waits for other streams.
 *
 * Errors: every call returns an hps_status; nothing is thrown across the ABI.
 * On failure *out handles are set to NULL and no memory is leaked.
 */
#ifndef HPS_GB300_H
#define HPS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st; /* cudaStream_t is `struct CUstream_st *` */

typedef enum {
  HPS_OK = 0,
  HPS_ERR_INVALID = -1,   /* bad argument: sizes, NULL pointers, q != p-2 ... */
  HPS_ERR_OOM = -2,       /* planned footprint exceeds free device memory   */
  HPS_ERR_SINGULAR = -3,  /* an exactly zero pivot in a leaf or merge LU     */
  HPS_ERR_CUDA = -4,      /* a CUDA runtime call failed                      */
  HPS_ERR_TIMEOUT = -5,   /* a bounded device-side wait gave up              */
  HPS_PENDING = 1         /* hps_server_poll: the request has not finished   */
} hps_status;

enum { HPS_DTN = 0, HPS_ITI = 1 };
enum { HPS_F64 = 0, HPS_C128 = 1 };

/* Tree over the box [lo, hi] (a square or cube: leaves must be cubes).
 * uniform_depth >= 0 selects the uniform tree of that depth (morton and level
 * must be NULL).  uniform_depth == -1 selects an adaptive octree (dim = 3,
 * DtN only, Section 4.2): n_leaves leaves, leaf n at level[n] (0..16) with
 * integer coordinates at that level encoded in morton[n] (bit 3b + a holds bit
 * b of the coordinate along axis a), listed depth first in Morton order
 * (the order hps_refine returns).  The leaves must tile the cube and be 2:1
 * balanced across faces; else HPS_ERR_INVALID.  For an adaptive tree a node's
 * boundary lists each face as the quadtree of its children's faces (Morton
 * order over the two tangential axes), each leaf panel q^2 points. */
typedef struct {
  int dim;                 /* 2 or 3 */
  double lo[3], hi[3];
  int uniform_depth;       /* L >= 0, or -1 for an adaptive octree */
  int64_t n_leaves;        /* 2^(dim L) for uniform trees */
  const uint64_t* morton;  /* adaptive: host array [n_leaves] */
  const int8_t* level;     /* adaptive: host array [n_leaves] */
} hps_tree;

/* Callback evaluating a function at n points (xyz: [n][3], host memory) into
 * out[n]; returns 0 on success.  ctx is the caller's pointer. */
typedef int (*hps_eval_fn)(void* ctx, int64_t n, const double* xyz, double* out);

/* Coefficients of L u = a Lap u + sum_k b_k d_k u + c u, each sampled at the
 * leaf nodes ([n_leaves][p^d] doubles).  NULL selects a = 1, b_k = 0, c = 0.
 * kind: HPS_DTN (2D or 3D, real data) or HPS_ITI (2D, complex data).
 * dtype must be HPS_F64 for HPS_DTN and HPS_C128 for HPS_ITI (coefficients
 * stay real in both; f, g and u follow dtype).  eta > 0 for HPS_ITI. */
typedef struct {
  int kind;
  int dtype;
  double eta;
  const double* a;
  const double* b[3];
  const double* c;
} hps_coeffs;

typedef struct {
  int version;          /* 1 */
  int want_root_map;    /* 1: also form the root's T and h (not needed to solve) */
  int profile;          /* 1: time every kernel launch with CUDA events (slower) */
  int lazy_root;        /* 1: keep the root's [C | h_int] and D's factors instead of
                           forming S = -D^{-1} C (Eq. "merge outputs 2"); each
                           solve then applies D^{-1} to C g + h_int.  Saves the
                           root's multi-RHS solve in hps_build; uniform and
                           adaptive trees, ignored with want_root_map.  With up to 8 right-hand
                           sides the root's triangular solves run as one
                           flag-ordered launch per triangle; if one of its
                           bounded waits gives up, that hps_solve (host u) or
                           the next one on the handle returns HPS_ERR_TIMEOUT. */
  int graph_solve;      /* 1: hps_solve / hps_solve_batched with device buffers on a
                           non-default stream replay a CUDA graph of the whole
                           solve (upward and downward passes), captured on the
                           second call with the same (nrhs, g, f, u) pointers;
                           up to 8 graphs per handle.  Uniform trees; ignored
                           while profiling.  The caller may change the data
                           behind the pointers between calls, not the pointers. */
  int iti_leaf;         /* ItI leaf solves: 0 automatic, 1 the complex LU of the whole
                           leaf matrix B = [G; L(I_i,:)] (Algorithm "2D ItI local
                           solve"), 2 elimination of the interior nodes (a real
                           LU of L(I_i,I_i) and a complex Schur complement on the
                           boundary nodes; same solution, about a third of the
                           flops).  Automatic takes 2 when the leaf Dirichlet
                           problem is far from resonance: max c <= min a * pi^2 /
                           (2 h^2) and max |b| h <= min a, h the leaf side. */
  int fp64_gemm;        /* 0: hps_build runs its large real and complex products
                           on the tensor cores as exact bf16 digit-slice
                           products (FP64 accuracy: operands cut into ten 6-bit
                           digits, the 55 digit products of weight above 2^-66
                           accumulated exactly and recombined in 64-bit
                           integers; it needs a transient device
                           workspace of up to about 1 GB, and a product whose
                           workspace cannot be allocated runs on the FP64
                           pipe); 1: every product on the FP64 pipe.  Solves
                           always use the FP64 pipe. */
  int recompute_budget_mb; /* > 0: device-memory budget (MiB) of the handle.  When the
                           planned footprint of a uniform tree (hps_plan_bytes)
                           exceeds it, the build keeps only the merges above the
                           largest complete subtrees that fit (each subtree's
                           root T and h, and device copies of the coefficients
                           and the source) and every hps_solve rebuilds each
                           subtree on its way down: Section 4.1, Algorithm
                           "our_recomputation", on the device.  Solves with a
                           new f also rebuild each subtree once per right-hand
                           side for its root's h.  Such a handle supports
                           hps_solve / hps_solve_batched only (not the adjoint,
                           hps_coeff_gradient, hps_solve_multi or
                           hps_solve_noalloc: HPS_ERR_INVALID); a singular pivot
                           inside a subtree is reported without the node.  If
                           no subtree depth fits, HPS_ERR_OOM.  0: off. */
} hps_options;

/* Kernel classes reported by hps_kernel_stats. */
enum {
  HPS_KCLASS_GEMM = 0,        /* batched / gathered FP64 or complex GEMM            */
  HPS_KCLASS_LU_PANEL = 1,    /* panel LU with partial pivoting                      */
  HPS_KCLASS_LASWP_TRSM = 2,  /* row interchanges + U12 triangular update            */
  HPS_KCLASS_TRSM_DIAG = 3,   /* diagonal-block triangular solves                    */
  HPS_KCLASS_ASSEMBLE = 4,    /* leaf operator assembly                              */
  HPS_KCLASS_GATHER = 5,      /* merge gathers, row permutations, scatters           */
  HPS_KCLASS_DOWN = 6,        /* downward-pass and leaf-output products              */
  HPS_KCLASS_OTHER = 7,       /* fills and copies                                    */
  HPS_KCLASS_GEMM_TC = 8,     /* FP64 / complex GEMM on the tensor cores (digit slices) */
  HPS_KCLASS_SPLIT = 9,       /* cutting GEMM operands into bf16 digit slices        */
  HPS_KCLASS_COUNT = 10
};

typedef struct {
  int64_t launches;  /* launches of this class in the last build or solve          */
  double flops;      /* algorithmic FP64 flops (complex multiply-add = 8)          */
  double ms;         /* summed CUDA-event time, or -1 when profiling is off         */
  double exec_flops; /* flops the executing pipe performs: the FP64 pipe's equal
                        flops except for the complex GEMM, which takes 3 real
                        products per complex multiply-add (Gauss / 3M form: 6
                        flops instead of 8); for HPS_KCLASS_GEMM_TC the bf16
                        tensor-core flops of the digit products over the padded
                        128 x 48 x 16 tiles (55 products per real product)    */
} hps_kernel_stat;

typedef struct hps_handle hps_handle;

/* Coordinates where the caller samples coefficients, f and g:
 * leaf_xyz: [n_leaves * p^d][dim] doubles (may be NULL),
 * bdry_xyz: [n_root_bdry][dim] doubles (may be NULL), both host memory.
 * n_root_bdry = 4 q 2^L (2D) or 6 q^2 4^L (3D).  Pure host computation.
 * Errors: HPS_ERR_INVALID for an unsupported tree, p < 4 or q != p - 2. */
hps_status hps_nodes(const hps_tree* tree, int p, int q, double* leaf_xyz, double* bdry_xyz);

/* Adaptive refinement (Section 4.2, Eq. "refinement check"): starting from
 * the uniform octree of depth min_depth over the cube [lo, hi], a leaf is
 * split while, for any of the n_fn functions, max |f(x1) - L_8f1 f(x0)| /
 * ||f||_inf >= eps, where x0 are its p^3 Chebyshev nodes, x1 the nodes of its
 * 8 children and L_8f1 the tensor interpolation between them (evaluated on
 * the device); ||f||_inf is the largest |f| over all points sampled up to
 * and including the current level.  Depth is capped at max_depth (<= 10).
 * The union of the functions' trees is then 2:1 balanced across faces.  The
 * functions are called on the host.  On return *n_leaves is the leaf count;
 * morton / level (host arrays) are filled when capacity >= *n_leaves, in the
 * order hps_tree expects.  HPS_ERR_INVALID for bad arguments or a failing
 * callback. */
hps_status hps_refine(const double lo[3], const double hi[3], int p, double eps, int min_depth,
                      int max_depth, int n_fn, const hps_eval_fn* fns, void* const* ctxs,
                      int64_t capacity, int64_t* n_leaves, uint64_t* morton, int8_t* level,
                      struct CUstream_st* stream);

/* Sizes that go with a tree: number of leaves, points per leaf and root
 * boundary points.  Any output pointer may be NULL. */
hps_status hps_sizes(const hps_tree* tree, int p, int q, int64_t* n_leaves,
                     int64_t* points_per_leaf, int64_t* n_root_bdry);

/* Build the solution operator (leaf stage + all merges).  f ([n_leaves][p^d],
 * real or complex per dtype) may be NULL (f = 0); it is the source used by
 * hps_solve(..., f = NULL, ...).  opts may be NULL (defaults).  On success
 * *out receives a new handle.  Errors: HPS_ERR_INVALID, HPS_ERR_OOM (before
 * any large allocation), HPS_ERR_SINGULAR (zero pivot; hps_last_error_detail
 * names the node), HPS_ERR_TIMEOUT, HPS_ERR_CUDA. */
hps_status hps_build(const hps_tree* tree, int p, int q, const hps_coeffs* coeffs,
                     const void* f, const hps_options* opts, struct CUstream_st* stream,
                     hps_handle** out);

/* Apply the solution operator: u = solution on all leaf nodes
 * ([n_leaves][p^d], dtype of the handle) for root boundary data g
 * ([n_root_bdry]).  f == NULL reuses the build-time source; otherwise the
 * upward particular pass (leaf and merge triangular solves with the stored
 * factors) runs for the new f first.  u must not alias g or f. */
hps_status hps_solve(hps_handle* h, const void* g, const void* f, void* u,
                     struct CUstream_st* stream);

/* nrhs independent right-hand sides at once: g is [nrhs][n_root_bdry],
 * f is NULL or [nrhs][n_leaves][p^d], u is [nrhs][n_leaves][p^d]. */
hps_status hps_solve_batched(hps_handle* h, int nrhs, const void* g, const void* f, void* u,
                             struct CUstream_st* stream);

/* Apply-only solves of n different operators at once (uniform trees; their
 * dimensions, kinds, depths and orders may all differ): for each i,
 * u[i] = solution of operator hs[i] for root data g[i] with the build-time
 * source, as hps_solve_batched(hs[i], nrhs[i], g[i], NULL, u[i]) computes it.
 * The downward passes share launches: one launch per tree level counted
 * from the roots serves every operator that has that level, and one launch
 * forms every leaf output (Section 3.4, Algorithm "down pass", over many
 * trees; the paper's remark that further sources cost only matrix-vector
 * products, Section 5.2).  Real and complex operators take separate
 * launches; a lazy root is applied per operator before the shared levels.
 *   hs: n distinct handles built on the current device;
 *   nrhs[i] >= 1; g[i]: [nrhs[i]][n_root_bdry_i], u[i]: [nrhs[i]][n_leaves_i]
 *   [p_i^d] device memory of the current device (dtype of hs[i]).
 * Each handle's previous work is waited for on `stream` first.  Results
 * equal hps_solve's up to rounding (the level products sum in another
 * order).  Errors: HPS_ERR_INVALID (n outside 1..1024, a NULL or repeated
 * handle, an adaptive handle, host buffers, another device), HPS_ERR_OOM
 * (a solve workspace), HPS_ERR_TIMEOUT, HPS_ERR_CUDA. */
hps_status hps_solve_multi(int n, hps_handle* const* hs, const int* nrhs, const void* const* g, void* const* u,
                           struct CUstream_st* stream);

/* Adjoint solve (uniform trees).  The solve is a linear map
 * u = A_g g + A_f f (Sections 3.2-3.4); this applies its conjugate
 * transpose with the stored factors, every step of the solve reversed:
 *   gbar = A_g^H ubar  ([nrhs][n_root_bdry], may be NULL),
 *   fbar = A_f^H ubar  ([nrhs][n_leaves][p^d], may be NULL; zero except at
 *                       each leaf's interior nodes),
 * for ubar [nrhs][n_leaves][p^d], so that Re<ubar, u> = Re<gbar, g> +
 * Re<fbar, f> for every (g, f).  fbar is the adjoint field of the leaf
 * collocation equations (input to hps_coeff_gradient).  Host or device
 * buffers as in hps_solve.  No counterpart in the paper, which computes
 * gradients by automatic differentiation of its JAX solver.
 * Errors: HPS_ERR_INVALID (adaptive handle, bad sizes), HPS_ERR_CUDA. */
hps_status hps_solve_adjoint(hps_handle* h, int nrhs, const void* ubar, void* gbar, void* fbar,
                             struct CUstream_st* stream);

/* Derivatives of Re<ubar, u> with respect to the coefficients at the leaf
 * interior nodes, from the solution u and the adjoint field fbar of
 * hps_solve_adjoint (same ubar), summed over the nrhs columns:
 *   gc = -Re(conj(fbar) u),  ga = -Re(conj(fbar) Lap u),
 *   gb[k] = -Re(conj(fbar) d_k u)  (derivatives of the leaf's spectral
 *   collocation, scaled to the leaf size);
 * every output is [n_leaves][p^d] doubles (gb: [dim][n_leaves][p^d]), zero
 * at leaf boundary nodes, and may be NULL.  u, fbar and the outputs must be
 * device memory.  Uniform trees. */
hps_status hps_coeff_gradient(hps_handle* h, int nrhs, const void* u, const void* fbar, double* ga,
                              double* gb, double* gc, struct CUstream_st* stream);

/* Release a handle (NULL is accepted).  Waits on the host for the handle's
 * own queued work (not for other work on the device) and returns its memory
 * to the library's stream-ordered pool, so a free never stalls unrelated
 * streams. */
void hps_free(hps_handle* h);

/* Batched dense product C = alpha A B + beta C (no counterpart in the paper:
 * the GEMM every merge and leaf stage of hps_build is made of, exposed so
 * that callers and tests can run it alone).  `batch` column-major matrices:
 * A item b at A + b*strideA (m x k, leading dimension lda), B item b at
 * B + b*strideB (k x n, ldb), C item b at C + b*strideC (m x n, ldc); strides
 * and leading dimensions in elements.  dtype HPS_F64 (double) or HPS_C128
 * (interleaved complex; alpha and beta are real).  mode 0: the tensor-core
 * digit-slice product that hps_build uses (operands cut into ten 6-bit bf16
 * digits per row of A / column of B, the 55 digit products whose digit
 * indices sum to at most 11 accumulated exactly in fp32, recombined in
 * 64-bit integers; for complex data the real and imaginary parts of a row /
 * column share one scale and each component of C is one accumulation of two
 * real products; a transient device workspace of up to about 1 GB); mode 1:
 * the FP64-pipe kernels.  Device pointers only; C must
 * not overlap A or B.  Enqueued on `stream` and synchronised before return.
 * HPS_ERR_INVALID for bad sizes, dtype or mode; HPS_ERR_OOM when device
 * memory cannot be allocated (mode 0 runs the product on the FP64 pipe when
 * its digit workspace does not fit); HPS_ERR_TIMEOUT when a bounded wait
 * inside the tensor-core kernel gave up (C is then undefined). */
hps_status hps_gemm(int dtype, int mode, int m, int n, int k, int batch, double alpha, const void* A, int lda,
                    int64_t strideA, const void* B, int ldb, int64_t strideB, double beta, void* C, int ldc,
                    int64_t strideC, struct CUstream_st* stream);

/* Batched LU factorisation with partial pivoting, in place (no counterpart in
 * the paper beyond the merge factor of D in Sec. 3.3 and the leaf
 * eliminations of Sec. 2.2-2.3, which the paper leaves to its library; this
 * is the factorisation hps_build runs there, exposed so that callers and
 * tests can run it alone).  `batch` column-major n x n matrices, item b at
 * A + b*strideA with leading dimension lda (elements); dtype HPS_F64 or
 * HPS_C128 (interleaved complex).  On return each item holds L (unit lower,
 * below the diagonal) and U (upper), and ipiv[b*n + j] (0-based) is the row
 * interchanged with row j at step j -- LAPACK's getrf convention, with the
 * same pivot choice: the largest magnitude (|re| + |im| for complex), and on
 * ties the lowest position in the row order reached so far.  info[b] = 0, or
 * the first column + 1 whose pivot is exactly zero.  mode 0: trailing
 * updates on the tensor cores where hps_build would put them; mode 1: FP64
 * pipe only.  Device pointers only (A, ipiv of batch*n ints, info of batch
 * ints); enqueued on `stream` and synchronised before return.
 * HPS_ERR_INVALID for bad sizes, dtype or mode; HPS_ERR_OOM when the
 * transient workspace cannot be allocated; HPS_ERR_TIMEOUT when a bounded
 * wait inside a kernel gave up (A is then undefined). */
hps_status hps_getrf(int dtype, int mode, int n, int batch, void* A, int lda, int64_t strideA, int* ipiv,
                     int* info, struct CUstream_st* stream);

/* Shape choices of the batched LU and of the product routing (no
 * counterpart in the paper, which factors and multiplies with its library).  Process-wide, read at each factorisation;
 * the defaults come from the autotuner's table (timed builds on GB300).
 *   HPS_TUNE_LU_BASE_PANELS_FEW  (0): recursive LU base width in panels for
 *       batches of fewer than 8 matrices (0: blocked right-looking);
 *   HPS_TUNE_LU_BASE_PANELS_MANY (1): the same for batches of 8 or more;
 *   HPS_TUNE_LU_FEW_MIN_N        (2): batches of fewer than 8 recurse only
 *       from this order on;
 *   HPS_TUNE_LU_CLUSTER_PANEL    (3): 1 factors tall panels in a thread-block
 *       cluster's distributed shared memory, 0 with cooperative groups;
 *   HPS_TUNE_TC_MIN_WORK_REAL    (4): a real product of the build runs on the
 *       tensor cores from M N K batch >= value x 1e5 on (hps_options.fp64_gemm
 *       = 0), else on the FP64 pipe;
 *   HPS_TUNE_TC_MIN_WORK_CPLX    (5): the same threshold for complex products;
 *   HPS_TUNE_TC_MIN_K            (6): products with an inner dimension below
 *       this stay on the FP64 pipe unless both M and N are at least 512;
 *   HPS_TUNE_TC_CHUNK_MB         (7): MiB of digit slices a batched tensor-core
 *       product cuts per launch group (the batch is cut into groups of items
 *       that fit; small groups are still in L2 when the products read them);
 *   HPS_TUNE_TC_PERSIST_MIN_K    (8): tensor-core products with an inner
 *       dimension of at least this run one CTA per SM that walks its tiles
 *       (copies and products of the next tile overlap the epilogue of the
 *       last), shorter ones one CTA per tile;
 *   HPS_TUNE_LU_PANEL_NB_FEW     (9): panel width (8 .. 32 columns; complex
 *       panels at most 16) of the LU of batches of fewer than 8 matrices.
 * Every choice gives the same pivots and results up to rounding.  Not to be
 * changed while a build runs.  HPS_ERR_INVALID for an unknown parameter or a
 * value outside 0 .. 2^20. */
enum { HPS_TUNE_LU_BASE_PANELS_FEW = 0, HPS_TUNE_LU_BASE_PANELS_MANY = 1, HPS_TUNE_LU_FEW_MIN_N = 2,
       HPS_TUNE_LU_CLUSTER_PANEL = 3, HPS_TUNE_TC_MIN_WORK_REAL = 4, HPS_TUNE_TC_MIN_WORK_CPLX = 5,
       HPS_TUNE_TC_MIN_K = 6, HPS_TUNE_TC_CHUNK_MB = 7, HPS_TUNE_TC_PERSIST_MIN_K = 8,
       HPS_TUNE_LU_PANEL_NB_FEW = 9 };
hps_status hps_tune_set(int param, int value);
hps_status hps_tune_get(int param, int* value);

/* Fault injection for tests (no counterpart in the paper).  Host side only:
 * no device fault, trap or hang is involved.  After hps_debug_fail_alloc(n)
 * with n > 0, the n-th device allocation of a handle (build buffers,
 * operators, solve workspaces) from then on fails as if cudaMalloc had
 * reported out-of-memory; the call that made it unwinds with HPS_ERR_OOM and
 * frees what it had allocated.  n <= 0 disarms.  hps_debug_alloc_count
 * returns the number of handle allocations made so far in this process. */
void hps_debug_fail_alloc(int64_t n);
int64_t hps_debug_alloc_count(void);

/* Bounded-wait check for tests (no counterpart in the paper).  Every wait
 * inside the library's kernels -- the inter-CTA barrier of the cooperative
 * panel LU (which = 0), the flag wait of the flag-ordered triangular solves
 * of a lazy root (which = 1) and the mbarrier wait of the tensor-core product
 * pipeline (which = 2) -- gives up after a bounded number of polls, records
 * a timeout in a device status word and lets its kernel end, so that a wait
 * that can never be satisfied costs an error status, not a hung GPU.  This
 * call runs the chosen wait in a one-CTA kernel on a word that nothing else
 * writes (satisfied = 0: the wait must run out) or on one already holding
 * the awaited value (satisfied = 1: the wait must pass at once), with at most
 * limit_polls polls (1 .. 2^24; the kernels' own limits are 2^22 to 2*10^7).
 * Returns HPS_ERR_TIMEOUT when the wait gave up, HPS_OK when it passed;
 * synchronises `stream`; uses 16 bytes of device memory for the call.
 * HPS_ERR_INVALID for a bad `which` or limit. */
hps_status hps_debug_wait_timeout(int which, int satisfied, int64_t limit_polls, struct CUstream_st* stream);

/* Static, NUL-terminated description of a status code. */
const char* hps_error_string(hps_status s);

/* Detail of the last error: for HPS_ERR_SINGULAR the leaf or merge-node id
 * (leaves: 0..n_leaves-1; then the merge nodes level by level from the
 * leaves up, in Morton order), else -1.  hps_build returns no handle on
 * failure, so pass h = NULL to read the detail of the calling thread's last
 * failed hps_build. */
hps_status hps_last_error_detail(hps_handle* h, int64_t* node);

/* Device bytes held by the handle (factors, operators, workspace). */
int64_t hps_device_bytes(const hps_handle* h);

/* Planned device bytes of a handle that hps_build would create for a uniform
 * tree (factors, operators and a one-right-hand-side solve workspace), before
 * building it: the figure a caller admits work by.  Pure host computation.
 * Not included: the transient digit-slice workspace of the tensor-core
 * products (hps_options.fp64_gemm = 0), at most about 1 GB while hps_build
 * runs and freed before it returns.  HPS_ERR_INVALID for adaptive trees and
 * bad arguments. */
hps_status hps_plan_bytes(const hps_tree* tree, int p, int q, int kind, int64_t* bytes);

/* Number of CUDA kernel launches issued by the last hps_build / hps_solve on h. */
int64_t hps_last_launch_count(const hps_handle* h);

/* Per-class launch count, algorithmic flops and (with profiling on) summed
 * kernel time of the last hps_build / hps_solve on h.  Synchronises the
 * handle's last stream when profiling is on.  HPS_ERR_INVALID for a bad class. */
hps_status hps_kernel_stats(hps_handle* h, int kclass, hps_kernel_stat* out);

/* Switch per-launch event timing on (1) or off (0) for later calls on h. */
hps_status hps_set_profiling(hps_handle* h, int on);

/* Per-launch trace of the last hps_build / hps_solve on h, recorded while
 * profiling is on (hps_options.profile or hps_set_profiling): one record per
 * library kernel launch, in launch order.  Shapes: GEMM m x n result with
 * inner dimension k; LU panel rows x panel width (k = CTAs per matrix);
 * row-interchange/U12 update panel width x trailing columns; diagonal
 * triangular solve block size x right-hand sides; 0 for other classes. */
typedef struct {
  int kclass;        /* HPS_KCLASS_*                                     */
  int m, n, k;       /* launch shape (see above)                         */
  int64_t batch;     /* matrices / merges / leaves in the launch         */
  double flops;      /* algorithmic flops of the launch                  */
  double ms;         /* CUDA-event time of the launch                    */
} hps_trace_rec;
/* Number of records (0 when profiling was off).  Synchronises the handle's
 * last stream.  HPS_ERR_INVALID for a NULL handle or pointer. */
hps_status hps_trace_count(hps_handle* h, int64_t* count);
/* Record i (0 <= i < count); HPS_ERR_INVALID when i is out of range. */
hps_status hps_trace_get(hps_handle* h, int64_t i, hps_trace_rec* out);

/* Allocation-free solve (uniform trees only; no counterpart in the paper; a service for callers
 * that cannot let the library allocate device memory at solve time: code
 * that works inside another allocator's memory budget, or that must not call
 * cudaMalloc / cudaFree there because those calls synchronise the device).
 * Same result as hps_solve(h, g, NULL, u, stream) -- downward pass and leaf
 * output with the build-time source -- but the per-level vectors live in one
 * static device array of 16 MiB that the library holds on every GPU that
 * loads it, until the process exits; no cudaMalloc, cudaFree or allocating
 * routine is called.
 *   g: [n_root_bdry] and u: [n_leaves][p^d] must be device memory.
 *   HPS_ERR_INVALID if g or u is host memory or memory of another device
 *   than the current one, if the handle was built on another device, if
 *   the handle keeps a lazy
 *   root (hps_options.lazy_root), or if the handle's downward
 *   pass needs more than the 16 MiB array (the sum over merge levels of
 *   n_merges x (interior unknowns + children's boundary points) elements,
 *   each rounded up to 256 bytes).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call shares the one array and leaves its
 * last contents there (nothing in it needs to start at zero): calls that
 * overlap on the GPU -- on different streams, or from different handles --
 * race on it and must be serialised by the caller. */
hps_status hps_solve_noalloc(hps_handle* h, const void* g, void* u, struct CUstream_st* stream);

#ifdef __cplusplus
}
#endif

#endif /* HPS_GB300_H */
