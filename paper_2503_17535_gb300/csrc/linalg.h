// Batched dense linear algebra on the device, FP64 and complex128.
//
// Column-major storage throughout.  A "batched operand" is either a device
// array of per-item base pointers (ptrs != nullptr) or a base pointer plus a
// fixed element stride between items; an element offset is then added to the
// item's base.  All launchers enqueue on `st` and return a cudaError_t from
// the launch check (nothing is synchronised here).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace hps {

// Kernel classes for launch / flop accounting and optional event timing.
enum KClass { K_GEMM = 0, K_LU_PANEL, K_LASWP_TRSM, K_TRSM_DIAG, K_ASSEMBLE, K_GATHER, K_DOWN,
              K_OTHER, K_GEMM_TC, K_SPLIT, K_COUNT };

// Launch accounting.  Every launch adds its class's algorithmic FP64 flops
// (a complex multiply-add counts 8); with `on` set each launch is also
// bracketed by CUDA events on its stream, summed by ms() after a sync.
struct Prof {
  bool on = false;
  int64_t launches = 0;
  int64_t n[K_COUNT] = {};
  double flops[K_COUNT] = {};  // algorithmic (complex multiply-add = 8)
  double exec[K_COUNT] = {};   // executed on the FP64 pipe (3M complex GEMM: 6 per multiply-add)
  std::vector<cudaEvent_t> ev[K_COUNT];
  cudaEvent_t pending = nullptr;
  // per-launch trace (profiling on): class, problem shape, flops and the
  // index of the launch's event pair in ev[cls]
  struct Rec { int cls, m, n, k; int64_t batch; double flops; int64_t ev; };
  std::vector<Rec> trace;
  int dims[4] = {0, 0, 0, 0};
  void begin(cudaStream_t st);
  // shape of the next launch (m x n result, inner dimension k, batch)
  void note(int m, int n, int k, int64_t batch) { dims[0] = m; dims[1] = n; dims[2] = k; dims[3] = (int)batch; }
  void end(int cls, double fl, cudaStream_t st, double executed = -1.0);
  double rec_ms(const Rec& r) const;
  void reset();
  double ms(int cls) const;
  ~Prof() { reset(); }
};

template <typename T>
struct BOp {
  T* const* ptrs = nullptr;  // per-item bases (device array) or nullptr
  T* base = nullptr;         // used when ptrs == nullptr
  int64_t stride = 0;        // elements between items when ptrs == nullptr
  int64_t off = 0;           // element offset added to every item's base
  int ld = 0;                // leading dimension (column-major)
  int div = 1;               // items b and b' share a base when b / div == b' / div
  int64_t sub = 0;           // extra stride for b % div (items inside one group)
  __host__ __device__ T* item(int b) const {
    return (ptrs ? ptrs[b] : base + (int64_t)(b / div) * stride + (int64_t)(b % div) * sub) + off;
  }
};

template <typename T>
BOp<T> bop(T* base, int64_t stride, int ld, int64_t off = 0) {
  BOp<T> o; o.base = base; o.stride = stride; o.ld = ld; o.off = off; return o;
}
template <typename T>
BOp<T> bopp(T* const* ptrs, int ld, int64_t off = 0) {
  BOp<T> o; o.ptrs = ptrs; o.ld = ld; o.off = off; return o;
}
template <typename T>
BOp<T> shifted(BOp<T> o, int64_t extra) { o.off += extra; return o; }
template <typename T>
BOp<T> grouped(BOp<T> o, int div) { o.div = div; return o; }

// Optional row/column index maps for gathered GEMM operands.  A map is an
// array [period][len]; batch item b uses row b % period.  nullptr = identity.
struct IMap {
  const int* idx = nullptr;
  int len = 0;      // entries per period row
  int period = 1;
  __device__ int at(int b, int i) const { return idx ? idx[(b % period) * len + i] : i; }
};

// C(crow(i), j) = alpha * sum_l A(arow(i), acol(l)) * B(brow(l), j) + beta * C(crow(i), j)
template <typename T>
struct GemmArgs {
  int M = 0, N = 0, K = 0, batch = 0;
  BOp<T> A, B, C;
  IMap arow, acol, brow, crow;
  T alpha = T(1.0), beta = T(0.0);
  // A enters conjugate-transposed: the (i, l) entry of the product's left
  // factor is conj(A(acol(l), arow(i))) (adjoint solves)
  bool ta = false;
  __device__ T a_at(const T* A, int b, int i, int l) const {
    if (!ta) return A[(int64_t)arow.at(b, i) + (int64_t)acol.at(b, l) * this->A.ld];
    return conj_of(A[(int64_t)acol.at(b, l) + (int64_t)arow.at(b, i) * this->A.ld]);
  }
};

template <typename T>
cudaError_t gemm(const GemmArgs<T>& g, cudaStream_t st, Prof* pf);

// Bounded-wait checks (hps_debug_wait_timeout): one CTA runs one of the
// library's bounded waits on a word nothing else writes (linalg.cu: the group
// barrier, which 0, and the triangular solves' flag wait, which 1, on the
// zeroed words[0..2]; gemm_tc.cu: the tensor-core pipeline's mbarrier wait).
cudaError_t debug_wait(int which, int satisfied, unsigned* words, unsigned long long limit, unsigned* err,
                       cudaStream_t st);
cudaError_t debug_mbar_wait(int satisfied, long limit, unsigned* err, cudaStream_t st);

// Tensor-core FP64 products (gemm_tc.cu): workspace for the operands' bf16
// digit slices.  gemm() routes a product to the tensor cores when the calling
// thread has an enabled workspace installed (TcScope) and the shape is large
// enough; otherwise it runs on the FP64 pipe.  Kernel timeouts set
// DEV_ERR_TIMEOUT in *err_slot.
struct TcWorkspace {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;  // stream the buffer was last allocated / used on
  unsigned* const* err_slot = nullptr;
  bool enabled = false;
  bool force = false;   // every product with K >= 1 (no size threshold)
};
TcWorkspace*& tc_workspace();
void tc_release(TcWorkspace* w);
// bytes the digit slices of one launch group may take (the allocation is at
// least 64 MB and at most this, unless a single matrix needs more)
size_t tc_workspace_cap();
struct TcScope {
  TcWorkspace* prev;
  explicit TcScope(TcWorkspace* w) : prev(tc_workspace()) { tc_workspace() = w; }
  ~TcScope() { tc_workspace() = prev; }
};
template <typename T>
bool tc_applicable(const GemmArgs<T>& g);
template <typename T>
cudaError_t gemm_tc(const GemmArgs<T>& g, cudaStream_t st, Prof* pf);

// Shape choices of the batched LU, process-wide (hps_tune_set / hps_tune_get
// expose them; the defaults are the values the autotuner measured best on
// GB300, csrc/tuned.h).
enum LuTuneParam {
  TUNE_LU_BASE_PANELS_FEW = 0,   // recursion base width in panels, batches < 8 (0: blocked)
  TUNE_LU_BASE_PANELS_MANY = 1,  // recursion base width in panels, batches >= 8
  TUNE_LU_FEW_MIN_N = 2,         // batches < 8 recurse only from this order on
  TUNE_LU_CLUSTER_PANEL = 3,     // 1: tall panels in a thread-block cluster, 0: cooperative groups
  TUNE_TC_MIN_WORK_REAL = 4,     // real products go to the tensor cores from M N K batch >= this x 1e5
  TUNE_TC_MIN_WORK_CPLX = 5,     // complex products: the same threshold
  TUNE_TC_MIN_K = 6,             // products with K below this stay on the FP64 pipe unless M, N >= 512
  TUNE_TC_CHUNK_MB = 7,          // digit slices of one launch group of a batched product, MiB
  TUNE_TC_PERSIST_MIN_K = 8,     // tensor-core products with K at least this walk their tiles persistently
  TUNE_LU_PANEL_NB_FEW = 9,      // panel width of the LU of batches of fewer than 8 matrices (8 .. 32)
  TUNE_COUNT = 10
};
int& lu_tune(int param);

// Streaming multiprocessors of the current device (queried once per process).
int device_sms();

struct LuWork {
  unsigned* bars = nullptr;   // 2 * batch barrier words (zeroed)
  void* pub = nullptr;        // publish buffer for G > 1
  size_t pub_bytes = 0;
};

template <typename T>
int lu_group_size(int n, int batch, int num_sms);

template <typename T>
size_t lu_pub_bytes(int n, int batch, int G);

// LU with partial pivoting of `batch` n x n matrices (in place), LAPACK
// semantics: ipiv[j] = row swapped with row j (0-based), perm = the row
// permutation P with P A = L U (perm[i] = original row of row i).
// G > 1 spreads each matrix over G co-resident CTAs (cooperative launch).
// ipiv/perm are int arrays of `batch * n` (item stride n).  info[b] = first
// zero-pivot column + 1 (0 if none).  dev_err receives DEV_ERR_* bits.
template <typename T>
cudaError_t getrf(BOp<T> A, int n, int batch, int* ipiv, int* perm, int* info, unsigned* dev_err,
                  int G, const LuWork& w, cudaStream_t st, Prof* pf);

// Solve (P^T L U) X = R in place for X given perm-gathered rows:
//   permute_rows: X(i, j) = R(perm[i], j)
//   getrs_inplace: X <- U^{-1} L^{-1} X
template <typename T>
cudaError_t permute_rows(BOp<T> src, BOp<T> dst, const int* perm, int n, int nrhs, int batch,
                         cudaStream_t st, Prof* pf);

template <typename T>
cudaError_t getrs_inplace(BOp<T> LU, int n, BOp<T> X, int nrhs, int batch, cudaStream_t st,
                          Prof* pf);

// One n x n LU factor against nrhs <= 8 columns (X <- U^{-1} L^{-1} X, X
// already row-permuted), each triangle in a single cooperative launch:
// 32-row blocks are solved in dependency order and published through
// per-block flags (flags[i] == epoch once block i is final).  The caller
// keeps one flag per 32 rows (device, initially 0) and a counter; each call
// uses two fresh epochs.  A wait that exceeds its poll limit stores 1 in
// *host_err (host-mapped memory) and the block goes on, so no launch hangs.
struct TrsvWork {
  unsigned* flags = nullptr;
  int nflags = 0;
  void* dinv = nullptr;        // 2 x nflags inverses of the 32 x 32 diagonal blocks (T)
  bool dinv_ready = false;     // formed on the first solve with the factor
  unsigned epoch = 0;
  volatile int* host_err = nullptr;  // host-mapped
  volatile int* dev_err = nullptr;   // its device alias
};

template <typename T>
bool trsv_flags_applicable(int n, int nrhs, int batch, const TrsvWork& w);

template <typename T>
cudaError_t getrs_flags(const T* LU, int n, int ld, T* X, int ldx, int nrhs, TrsvWork& w, cudaStream_t st,
                        Prof* pf);

// Conjugate transposes for the adjoint solves: dst(perm[i], j) = src(i, j),
// and X <- (U^H)^{-1} then (L^H)^{-1} with the LU factors of getrf (the
// caller applies the inverse row permutation afterwards).
template <typename T>
cudaError_t permute_rows_inv(BOp<T> src, BOp<T> dst, const int* perm, int n, int nrhs, int batch,
                             cudaStream_t st);
template <typename T>
cudaError_t getrs_h(BOp<T> LU, int n, BOp<T> X, int nrhs, int batch, cudaStream_t st, Prof* pf);

// C = alpha * C + beta (identity added on the diagonal when diag != 0) helpers
template <typename T>
cudaError_t fill(BOp<T> C, int M, int N, int batch, T value, T diag, cudaStream_t st, Prof* pf);

}  // namespace hps
