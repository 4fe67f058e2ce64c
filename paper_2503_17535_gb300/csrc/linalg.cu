// Batched FP64 / complex128 dense kernels: gathered GEMM, panel LU with
// partial pivoting (one CTA per matrix, a thread-block cluster per matrix,
// or a cooperative group of CTAs per matrix), row interchanges + triangular
// update, recursive LU and triangular solves, and flag-ordered solves of a
// single large factor.
//
// GB300 has about 1 TFLOP/s of FP64 (2 DFMA per clock per SM), so every
// kernel here is bound by the FP64 pipe long before HBM or shared memory:
// the designs aim at keeping all 152 SMs issuing FMAs (enough CTAs per level,
// clusters or cooperative groups for single large matrices), at spending no
// FP64 instruction that is not part of the algorithm, and at keeping FP64
// latency chains (a reciprocal, a serial load) off the per-column critical
// path of the panels.
#include "linalg.h"

#include <cooperative_groups.h>

#include <algorithm>
#include <cstdio>

namespace hps {

void Prof::begin(cudaStream_t st) {
  if (!on) return;
  cudaEventCreate(&pending);
  cudaEventRecord(pending, st);
}

void Prof::end(int cls, double fl, cudaStream_t st, double executed) {
  ++launches;
  ++n[cls];
  flops[cls] += fl;
  exec[cls] += executed < 0.0 ? fl : executed;
  if (!on || !pending) {
    dims[0] = dims[1] = dims[2] = dims[3] = 0;
    return;
  }
  cudaEvent_t e1;
  cudaEventCreate(&e1);
  cudaEventRecord(e1, st);
  trace.push_back(Rec{cls, dims[0], dims[1], dims[2], dims[3], fl, (int64_t)ev[cls].size()});
  dims[0] = dims[1] = dims[2] = dims[3] = 0;
  ev[cls].push_back(pending);
  ev[cls].push_back(e1);
  pending = nullptr;
}

double Prof::rec_ms(const Rec& r) const {
  float m = 0.f;
  if (r.ev + 1 < (int64_t)ev[r.cls].size() &&
      cudaEventElapsedTime(&m, ev[r.cls][r.ev], ev[r.cls][r.ev + 1]) == cudaSuccess)
    return m;
  return -1.0;
}

void Prof::reset() {
  for (int c = 0; c < K_COUNT; ++c) {
    for (cudaEvent_t e : ev[c]) cudaEventDestroy(e);
    ev[c].clear();
    n[c] = 0;
    flops[c] = 0.0;
    exec[c] = 0.0;
  }
  if (pending) cudaEventDestroy(pending);
  pending = nullptr;
  launches = 0;
  trace.clear();
}

double Prof::ms(int cls) const {
  double t = 0.0;
  for (size_t i = 0; i + 1 < ev[cls].size(); i += 2) {
    float m = 0.f;
    if (cudaEventElapsedTime(&m, ev[cls][i], ev[cls][i + 1]) == cudaSuccess) t += m;
  }
  return t;
}

template <typename T> constexpr double fma_flops() { return 2.0; }
template <> constexpr double fma_flops<cplx>() { return 8.0; }

// ---------------------------------------------------------------- GEMM ----

// Tile shapes: 64 x 64 (4 x 4 outputs per thread) for large FP64 products,
// 32 x 32 (2 x 2 per thread) where 64-wide tiles would leave much of the
// last tile row / column empty (the leaf updates of (p-2)^2-sized blocks).
template <typename T, int WIDE> struct GemmTile;
template <> struct GemmTile<double, 1> { enum { BM = 64, BN = 64, BK = 16, TM = 4, TN = 4 }; };
template <> struct GemmTile<double, 0> { enum { BM = 32, BN = 32, BK = 16, TM = 2, TN = 2 }; };
template <> struct GemmTile<cplx, 1> { enum { BM = 32, BN = 32, BK = 16, TM = 2, TN = 2 }; };
template <> struct GemmTile<cplx, 0> { enum { BM = 32, BN = 32, BK = 16, TM = 2, TN = 2 }; };

// Epilogue modes: the LU / TRSM / Schur updates are C <- C - A B and the
// leaf products C <- A B; handling those two forms apart keeps the general
// alpha / beta arithmetic (a complex multiply and multiply-add per element)
// off the FP64 pipe, where it costs as much as several steps of K.
enum { EPI_GENERAL = 0, EPI_SUB = 1, EPI_SET = 2 };

template <typename T>
inline int epi_mode(const GemmArgs<T>& g) {
  if (g.alpha == T(-1.0) && g.beta == T(1.0)) return EPI_SUB;
  if (g.alpha == T(1.0) && is_zero(g.beta)) return EPI_SET;
  return EPI_GENERAL;
}

template <typename T, int MODE, int WIDE>
__global__ void __launch_bounds__(256) k_gemm(GemmArgs<T> g) {
  constexpr int BM = GemmTile<T, WIDE>::BM, BN = GemmTile<T, WIDE>::BN, BK = GemmTile<T, WIDE>::BK;
  constexpr int TM = GemmTile<T, WIDE>::TM, TN = GemmTile<T, WIDE>::TN;
  constexpr int RX = BM / TM;  // threads along M (16)
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % RX, ty = tid / RX;
  for (int b = blockIdx.z; b < g.batch; b += gridDim.z) {
    const T* A = g.A.item(b);
    const T* B = g.B.item(b);
    T* C = g.C.item(b);
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    T acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        acc[r][c] = T(0.0);
        if (MODE == EPI_SUB) {
          const int gi = i0 + tx + RX * r, gj = j0 + ty + (256 / RX) * c;
          if (gi < g.M && gj < g.N) acc[r][c] = C[(int64_t)g.crow.at(b, gi) + (int64_t)gj * g.C.ld];
        }
      }
    for (int k0 = 0; k0 < g.K; k0 += BK) {
      for (int e = tid; e < BM * BK; e += 256) {
        int i = e % BM, l = e / BM;
        int gi = i0 + i, gl = k0 + l;
        T v = T(0.0);
        if (gi < g.M && gl < g.K)
          v = A[(int64_t)g.arow.at(b, gi) + (int64_t)g.acol.at(b, gl) * g.A.ld];
        As[l][i] = v;
      }
      for (int e = tid; e < BK * BN; e += 256) {
        int l = e % BK, j = e / BK;
        int gl = k0 + l, gj = j0 + j;
        T v = T(0.0);
        if (gl < g.K && gj < g.N) v = B[(int64_t)g.brow.at(b, gl) + (int64_t)gj * g.B.ld];
        Bs[l][j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T av[TM], bv[TN];
#pragma unroll
        for (int r = 0; r < TM; ++r) av[r] = As[kk][tx + RX * r];
#pragma unroll
        for (int c = 0; c < TN; ++c) bv[c] = Bs[kk][ty + (256 / RX) * c];
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
          for (int c = 0; c < TN; ++c)
            acc[r][c] = MODE == EPI_SUB ? fmsc(acc[r][c], av[r], bv[c]) : fmac(acc[r][c], av[r], bv[c]);
      }
      __syncthreads();
    }
    const bool use_beta = !is_zero(g.beta);
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      int gi = i0 + tx + RX * r;
      if (gi >= g.M) continue;
      int64_t ci = g.crow.at(b, gi);
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        int gj = j0 + ty + (256 / RX) * c;
        if (gj >= g.N) continue;
        T* p = C + ci + (int64_t)gj * g.C.ld;
        if (MODE != EPI_GENERAL) {
          *p = acc[r][c];
        } else {
          T v = g.alpha * acc[r][c];
          if (use_beta) v = fmac(v, g.beta, *p);
          *p = v;
        }
      }
    }
  }
}

// Complex GEMM by the 3M method: with A = Ar + i Ai and B = Br + i Bi, the
// real products P1 = Ar Br, P2 = Ai Bi and P3 = (Ar + Ai)(Br + Bi) give
// C = (P1 - P2) + i (P3 - P1 - P2).  Each complex multiply-add costs three
// real FMAs instead of four on the FP64 pipe; the sums Ar + Ai and Br + Bi
// are formed once per element when the tile is staged in shared memory.
// With MODE == EPI_SUB the accumulators start from C so that the update
// needs three additions per element: p1 = 0, p2 = Re C, p3 = Re C - Im C give
// Re(C - AB) = p2 - p1 and Im(C - AB) = p1 + p2 - p3 after the products.
template <int MODE>
__global__ void __launch_bounds__(256) k_gemm_c3m(GemmArgs<cplx> g) {
  constexpr int BM = 32, BN = 32, BK = 16, TM = 2, TN = 2, RX = 16;
  __shared__ double Ar[BK][BM], Ai[BK][BM], As[BK][BM];
  __shared__ double Br[BK][BN], Bi[BK][BN], Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % RX, ty = tid / RX;
  for (int b = blockIdx.z; b < g.batch; b += gridDim.z) {
    const cplx* A = g.A.item(b);
    const cplx* B = g.B.item(b);
    cplx* C = g.C.item(b);
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    double p1[TM][TN], p2[TM][TN], p3[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        p1[r][c] = p2[r][c] = p3[r][c] = 0.0;
        if (MODE == EPI_SUB) {
          const int gi = i0 + tx + RX * r, gj = j0 + ty + 16 * c;
          if (gi < g.M && gj < g.N) {
            const cplx cv = C[(int64_t)g.crow.at(b, gi) + (int64_t)gj * g.C.ld];
            p2[r][c] = cv.re;
            p3[r][c] = cv.re - cv.im;
          }
        }
      }
    for (int k0 = 0; k0 < g.K; k0 += BK) {
      for (int e = tid; e < BM * BK; e += 256) {
        const int i = e % BM, l = e / BM;
        const int gi = i0 + i, gl = k0 + l;
        cplx v(0.0, 0.0);
        if (gi < g.M && gl < g.K) v = A[(int64_t)g.arow.at(b, gi) + (int64_t)g.acol.at(b, gl) * g.A.ld];
        Ar[l][i] = v.re; Ai[l][i] = v.im; As[l][i] = v.re + v.im;
      }
      for (int e = tid; e < BK * BN; e += 256) {
        const int l = e % BK, j = e / BK;
        const int gl = k0 + l, gj = j0 + j;
        cplx v(0.0, 0.0);
        if (gl < g.K && gj < g.N) v = B[(int64_t)g.brow.at(b, gl) + (int64_t)gj * g.B.ld];
        Br[l][j] = v.re; Bi[l][j] = v.im; Bs[l][j] = v.re + v.im;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double ar[TM], ai[TM], as[TM], br[TN], bi[TN], bs[TN];
#pragma unroll
        for (int r = 0; r < TM; ++r) { ar[r] = Ar[kk][tx + RX * r]; ai[r] = Ai[kk][tx + RX * r]; as[r] = As[kk][tx + RX * r]; }
#pragma unroll
        for (int c = 0; c < TN; ++c) { br[c] = Br[kk][ty + 16 * c]; bi[c] = Bi[kk][ty + 16 * c]; bs[c] = Bs[kk][ty + 16 * c]; }
#pragma unroll
        for (int r = 0; r < TM; ++r)
#pragma unroll
          for (int c = 0; c < TN; ++c) {
            p1[r][c] = fma(ar[r], br[c], p1[r][c]);
            p2[r][c] = fma(ai[r], bi[c], p2[r][c]);
            p3[r][c] = fma(as[r], bs[c], p3[r][c]);
          }
      }
      __syncthreads();
    }
    const bool use_beta = !is_zero(g.beta);
#pragma unroll
    for (int r = 0; r < TM; ++r) {
      const int gi = i0 + tx + RX * r;
      if (gi >= g.M) continue;
      const int64_t ci = g.crow.at(b, gi);
#pragma unroll
      for (int c = 0; c < TN; ++c) {
        const int gj = j0 + ty + 16 * c;
        if (gj >= g.N) continue;
        cplx* p = C + ci + (int64_t)gj * g.C.ld;
        if (MODE == EPI_SUB) {
          *p = cplx(p2[r][c] - p1[r][c], (p1[r][c] + p2[r][c]) - p3[r][c]);
        } else if (MODE == EPI_SET) {
          *p = cplx(p1[r][c] - p2[r][c], p3[r][c] - (p1[r][c] + p2[r][c]));
        } else {
          const cplx acc(p1[r][c] - p2[r][c], p3[r][c] - p1[r][c] - p2[r][c]);
          cplx v = g.alpha * acc;
          if (use_beta) v = fmac(v, g.beta, *p);
          *p = v;
        }
      }
    }
  }
}

template <typename T> struct UseC3M { static constexpr bool value = false; };
template <> struct UseC3M<cplx> { static constexpr bool value = true; };

// Skinny variant for N <= 8 right-hand sides (the solve path): one thread
// per output row, B chunks staged in shared memory, A read column by column
// (coalesced along the rows).  NC is the column count rounded up to 1, 2, 4
// or 8: the FP64 pipe spends its cycles on predicated-off FMAs too, so the
// kernel never carries more columns than it needs.
template <typename T, int NC>
__global__ void __launch_bounds__(128) k_gemm_skinny(GemmArgs<T> g) {
  constexpr int KC = 32;
  __shared__ T Bs[KC][NC];
  const int tid = threadIdx.x;
  for (int b = blockIdx.z; b < g.batch; b += gridDim.z) {
    const T* A = g.A.item(b);
    const T* B = g.B.item(b);
    T* C = g.C.item(b);
    const int i = blockIdx.x * 128 + tid;
    const bool act = i < g.M;
    const int64_t ar = act ? g.arow.at(b, i) : 0;
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = T(0.0);
    for (int k0 = 0; k0 < g.K; k0 += KC) {
      const int kc = min(KC, g.K - k0);
      __syncthreads();
      for (int e = tid; e < KC * NC; e += 128) {
        const int l = e % KC, c = e / KC;
        Bs[l][c] = (l < kc && c < g.N) ? B[(int64_t)g.brow.at(b, k0 + l) + (int64_t)c * g.B.ld] : T(0.0);
      }
      __syncthreads();
      if (act) {
        if (kc == KC) {
          // full chunk: unrolled so that several column loads are in flight
#pragma unroll 8
          for (int l = 0; l < KC; ++l) {
            const T a = A[ar + (int64_t)g.acol.at(b, k0 + l) * g.A.ld];
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = fmac(acc[c], a, Bs[l][c]);
          }
        } else {
          for (int l = 0; l < kc; ++l) {
            const T a = A[ar + (int64_t)g.acol.at(b, k0 + l) * g.A.ld];
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[c] = fmac(acc[c], a, Bs[l][c]);
          }
        }
      }
    }
    if (act) {
      const int64_t ci = g.crow.at(b, i);
      const bool use_beta = !is_zero(g.beta);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (c >= g.N) break;
        T* p = C + ci + (int64_t)c * g.C.ld;
        T v = g.alpha * acc[c];
        if (use_beta) v = fmac(v, g.beta, *p);
        *p = v;
      }
    }
  }
}

// Skinny product with few rows in the whole launch (the top levels of the
// solve): 32 rows x 8 groups of the inner dimension per CTA, the 8 partial
// sums added in shared memory in a fixed order.
template <typename T, int NC>
__global__ void __launch_bounds__(256) k_gemm_skinny_kg(GemmArgs<T> g) {
  __shared__ T part[8][NC][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int b = blockIdx.z; b < g.batch; b += gridDim.z) {
    const T* A = g.A.item(b);
    const T* B = g.B.item(b);
    T* C = g.C.item(b);
    const int i = blockIdx.x * 32 + lane;
    const bool act = i < g.M;
    const int64_t ar = act ? g.arow.at(b, i) : 0;
    T acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = T(0.0);
    if (act) {
#pragma unroll 4
      for (int l = w; l < g.K; l += 8) {
        const T a = A[ar + (int64_t)g.acol.at(b, l) * g.A.ld];
        const int64_t br = g.brow.at(b, l);
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (c < g.N) acc[c] = fmac(acc[c], a, B[br + (int64_t)c * g.B.ld]);
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) part[w][c][lane] = acc[c];
    __syncthreads();
    if (w == 0 && act) {
      const int64_t ci = g.crow.at(b, i);
      const bool use_beta = !is_zero(g.beta);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (c >= g.N) break;
        T v = part[0][c][lane];
        for (int k = 1; k < 8; ++k) v = v + part[k][c][lane];
        T* p = C + ci + (int64_t)c * g.C.ld;
        v = g.alpha * v;
        if (use_beta) v = fmac(v, g.beta, *p);
        *p = v;
      }
    }
    __syncthreads();
  }
}

// Products with a conjugate-transposed left factor (the adjoint solves):
// 32 x 32 output tiles, 16-deep slabs of both operands staged in shared
// memory.  Kept apart from the forward kernels so that their code is not
// touched by the transposed operand access.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_ta(GemmArgs<T> g) {
  constexpr int BM = 32, BN = 32, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;  // 2 x 2 outputs per thread
  for (int b = blockIdx.z; b < g.batch; b += gridDim.z) {
    const T* A = g.A.item(b);
    const T* B = g.B.item(b);
    T* C = g.C.item(b);
    const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
    T acc[2][2];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) acc[r][c] = T(0.0);
    for (int k0 = 0; k0 < g.K; k0 += BK) {
      for (int e = tid; e < BM * BK; e += 256) {
        const int l = e % BK, i = e / BK;  // consecutive threads walk A's column
        const int gi = i0 + i, gl = k0 + l;
        As[l][i] = (gi < g.M && gl < g.K) ? g.a_at(A, b, gi, gl) : T(0.0);
      }
      for (int e = tid; e < BK * BN; e += 256) {
        const int l = e % BK, j = e / BK;
        const int gl = k0 + l, gj = j0 + j;
        Bs[l][j] = (gl < g.K && gj < g.N) ? B[(int64_t)g.brow.at(b, gl) + (int64_t)gj * g.B.ld] : T(0.0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        const T a0 = As[kk][tx], a1 = As[kk][tx + 16], b0 = Bs[kk][ty], b1 = Bs[kk][ty + 16];
        acc[0][0] = fmac(acc[0][0], a0, b0);
        acc[0][1] = fmac(acc[0][1], a0, b1);
        acc[1][0] = fmac(acc[1][0], a1, b0);
        acc[1][1] = fmac(acc[1][1], a1, b1);
      }
      __syncthreads();
    }
    const bool use_beta = !is_zero(g.beta);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int gi = i0 + tx + 16 * r;
      if (gi >= g.M) continue;
      const int64_t ci = g.crow.at(b, gi);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int gj = j0 + ty + 16 * c;
        if (gj >= g.N) continue;
        T* p = C + ci + (int64_t)gj * g.C.ld;
        T v = g.alpha * acc[r][c];
        if (use_beta) v = fmac(v, g.beta, *p);
        *p = v;
      }
    }
  }
}

// Wide (64 x 64) tiles unless they leave more than 1/8 of the computed
// outputs empty where 32 x 32 tiles would not: the padded area decides.
inline bool wide_tiles(int M, int N, int BM, int BN) {
  if (BM == 32) return false;
  auto padded = [](int n, int b) { return (double)((n + b - 1) / b) * b; };
  const double wide = padded(M, BM) * padded(N, BN), narrow = padded(M, 32) * padded(N, 32);
  return wide <= 1.125 * narrow;
}

template <typename T>
cudaError_t gemm(const GemmArgs<T>& g, cudaStream_t st, Prof* pf) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.K > 0 && tc_applicable(g)) {
    const cudaError_t e = gemm_tc(g, st, pf);
    if (e != cudaErrorMemoryAllocation) return e;
    // the digit-slice workspace could not grow (nothing was launched): the
    // product runs on the FP64 pipe instead
    cudaGetLastError();
  }
  constexpr int BM = GemmTile<T, 1>::BM, BN = GemmTile<T, 1>::BN;
  if (pf) {
    pf->begin(st);
    pf->note(g.M, g.N, g.K, g.batch);
  }
  if (g.ta) {
    dim3 grid((g.M + 31) / 32, (g.N + 31) / 32, std::min(g.batch, 65535));
    k_gemm_ta<T><<<grid, 256, 0, st>>>(g);
  } else if (g.N <= 8 && g.K >= 128 && (int64_t)((g.M + 127) / 128) * g.batch < 304) {
    dim3 grid((g.M + 31) / 32, 1, std::min(g.batch, 65535));
    if (g.N == 1) k_gemm_skinny_kg<T, 1><<<grid, 256, 0, st>>>(g);
    else if (g.N == 2) k_gemm_skinny_kg<T, 2><<<grid, 256, 0, st>>>(g);
    else if (g.N <= 4) k_gemm_skinny_kg<T, 4><<<grid, 256, 0, st>>>(g);
    else k_gemm_skinny_kg<T, 8><<<grid, 256, 0, st>>>(g);
  } else if (g.N <= 8) {
    dim3 grid((g.M + 127) / 128, 1, std::min(g.batch, 65535));
    if (g.N == 1) k_gemm_skinny<T, 1><<<grid, 128, 0, st>>>(g);
    else if (g.N == 2) k_gemm_skinny<T, 2><<<grid, 128, 0, st>>>(g);
    else if (g.N <= 4) k_gemm_skinny<T, 4><<<grid, 128, 0, st>>>(g);
    else k_gemm_skinny<T, 8><<<grid, 128, 0, st>>>(g);
  } else if (UseC3M<T>::value) {
    dim3 grid((g.M + 31) / 32, (g.N + 31) / 32, std::min(g.batch, 65535));
    const GemmArgs<cplx>& gc = *reinterpret_cast<const GemmArgs<cplx>*>(&g);
    switch (epi_mode(gc)) {
      case EPI_SUB: k_gemm_c3m<EPI_SUB><<<grid, 256, 0, st>>>(gc); break;
      case EPI_SET: k_gemm_c3m<EPI_SET><<<grid, 256, 0, st>>>(gc); break;
      default: k_gemm_c3m<EPI_GENERAL><<<grid, 256, 0, st>>>(gc); break;
    }
    const double mnk = g.M * (double)g.N * g.K * g.batch;
    if (pf) pf->end(K_GEMM, 8.0 * mnk, st, 6.0 * mnk);
    return cudaGetLastError();
  } else if (wide_tiles(g.M, g.N, BM, BN)) {
    dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, std::min(g.batch, 65535));
    switch (epi_mode(g)) {
      case EPI_SUB: k_gemm<T, EPI_SUB, 1><<<grid, 256, 0, st>>>(g); break;
      case EPI_SET: k_gemm<T, EPI_SET, 1><<<grid, 256, 0, st>>>(g); break;
      default: k_gemm<T, EPI_GENERAL, 1><<<grid, 256, 0, st>>>(g); break;
    }
  } else {
    dim3 grid((g.M + 31) / 32, (g.N + 31) / 32, std::min(g.batch, 65535));
    switch (epi_mode(g)) {
      case EPI_SUB: k_gemm<T, EPI_SUB, 0><<<grid, 256, 0, st>>>(g); break;
      case EPI_SET: k_gemm<T, EPI_SET, 0><<<grid, 256, 0, st>>>(g); break;
      default: k_gemm<T, EPI_GENERAL, 0><<<grid, 256, 0, st>>>(g); break;
    }
  }
  if (pf) pf->end(K_GEMM, fma_flops<T>() * g.M * (double)g.N * g.K * g.batch, st);
  return cudaGetLastError();
}

// --------------------------------------------------------------- fill -----

template <typename T>
__global__ void k_fill(BOp<T> C, int M, int N, int batch, T value, T diag) {
  int64_t total = (int64_t)M * N;
  for (int b = blockIdx.y; b < batch; b += gridDim.y) {
    T* c = C.item(b);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      int i = (int)(e % M), j = (int)(e / M);
      c[i + (int64_t)j * C.ld] = (i == j) ? diag : value;
    }
  }
}

template <typename T>
cudaError_t fill(BOp<T> C, int M, int N, int batch, T value, T diag, cudaStream_t st, Prof* pf) {
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  int64_t total = (int64_t)M * N;
  int bx = (int)std::min<int64_t>((total + 255) / 256, 4096);
  dim3 grid(bx, std::min(batch, 65535));
  if (pf) pf->begin(st);
  k_fill<T><<<grid, 256, 0, st>>>(C, M, N, batch, value, diag);
  if (pf) pf->end(K_OTHER, 0.0, st);
  return cudaGetLastError();
}

// Streaming multiprocessors of the current device (queried once per process).
int device_sms() {
  static const int sms = [] {
    int dev = 0, s = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return 1;
    }
    return s > 0 ? s : 1;
  }();
  return sms;
}

// whole-warp shuffle of a real or complex value
__device__ inline double shfl_val(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ inline cplx shfl_val(cplx v, int src) {
  return cplx(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}

// ------------------------------------------------------------ panel LU ----

// Factor the panel A[k0:n, k0:k0+nb) of each matrix with partial pivoting.
// The rows [k0, n) are split into G contiguous chunks, one per CTA of the
// matrix's group; each CTA holds its chunk of the panel in shared memory
// (column-major, `ch` rows).  Per column: local argmax, publish candidate,
// group barrier, global pick (largest |.|, lowest row on ties), swap, update.
// Pivot order: larger magnitude first, then the lower row.  Magnitudes are
// non-negative (or -1 for "none"), so their IEEE bit patterns order like the
// values as signed 64-bit integers; comparing those keeps the search on the
// integer pipe instead of the FP64 pipe.
__device__ __forceinline__ bool piv_better(double m, int r, double best_m, int best_r) {
  const long long a = __double_as_longlong(m), b = __double_as_longlong(best_m);
  return a > b || (a == b && r < best_r);
}

// The panel rows [r0, r0 + rc) x columns [k0, k0 + nb) into shared memory
// (column-major, ch rows) with asynchronous copies: every load is in flight
// at once (plain loads would wait one by one, since the compiler cannot tell
// the global source from the shared destination).  Ends with the copies done
// for this thread; the caller's barrier publishes them.
template <typename T>
__device__ __forceinline__ void load_panel(T* Ps, const T* Ab, int lda, int r0, int k0, int rc, int ch, int nb,
                                           int tid, int nth) {
  for (int c = 0; c < nb; ++c)
    for (int r = tid; r < rc; r += nth)
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((unsigned)__cvta_generic_to_shared(
                       Ps + r + (size_t)c * ch)),
                   "l"(Ab + (int64_t)(r0 + r) + (int64_t)(k0 + c) * lda), "n"((int)sizeof(T))
                   : "memory");
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_all;" ::: "memory");
}

template <typename T, bool COOP>
__global__ void __launch_bounds__(256) k_lu_panel(BOp<T> A, int n, int k0, int nb, int G, int* ipiv,
                                                  int* info, unsigned* bars, T* pubv, double* pubm,
                                                  int* pubr, unsigned* dev_err) {
  // Threads form RT row lanes x CT column lanes (CT > 1 when the chunk has
  // fewer rows than threads); per column the pivot is reduced (warp
  // shuffles, then every thread over the warp results), rows j and p are
  // swapped one column per thread, every thread forms the multipliers of its
  // rows, and after one more barrier updates its columns (cyclic from
  // jj + 1), the lane of column jj + 1 tracking that column's largest entry
  // for the next step: three block barriers per column.
  extern __shared__ unsigned char smem_raw[];
  T* Ps = reinterpret_cast<T*>(smem_raw);
  const int b = blockIdx.x / G, g = blockIdx.x % G;
  const int rows = n - k0;
  const int ch = (rows + G - 1) / G;
  const int r0 = k0 + g * ch;                 // first global row of this chunk
  const int rc = max(0, min(ch, n - r0));     // rows in this chunk
  T* Ab = A.item(b);
  const int lda = A.ld;
  T* Wv = Ps + (size_t)ch * nb;               // pivot row after the swap (nb)
  T* Rv = Wv + nb;                            // old row j (nb)
  __shared__ double red_m[8];
  __shared__ int red_r[8];
  __shared__ int s_bg;
  __shared__ double s_inv_raw[2];  // 1 / pivot, formed once per column
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nth >> 5;
  int CT = 1;
  while (CT < 16 && CT * 2 <= nb && (nth / (CT * 2)) >= rc && nth / (CT * 2) >= 32) CT *= 2;
  const int RT = nth / CT, rt = tid % RT, ct = tid / RT;

  load_panel(Ps, Ab, lda, r0, k0, rc, ch, nb, tid, nth);
  __syncthreads();
  T* pv = COOP ? pubv + (size_t)b * 2 * (G + 1) * nb : nullptr;
  double* pm = COOP ? pubm + (size_t)b * 2 * G : nullptr;
  int* pr = COOP ? pubr + (size_t)b * 2 * G : nullptr;
  unsigned* bar = COOP ? bars + 2 * b : nullptr;

  // this thread's best entry of the current column (rows >= j)
  double best = -1.0;
  int brow = 0x7fffffff;
  for (int r = max(0, k0 - r0) + tid; r < rc; r += nth) {
    const double m = mag1(Ps[r]);
    if (piv_better(m, r0 + r, best, brow)) { best = m; brow = r0 + r; }
  }
  for (int jj = 0; jj < nb; ++jj) {
    const int j = k0 + jj;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double m2 = __shfl_down_sync(0xffffffffu, best, o);
      const int r2 = __shfl_down_sync(0xffffffffu, brow, o);
      if (piv_better(m2, r2, best, brow)) { best = m2; brow = r2; }
    }
    if (lane == 0) { red_m[wid] = best; red_r[wid] = brow; }
    __syncthreads();
    double pmag = red_m[0];
    int p = red_r[0];
    for (int w = 1; w < nw; ++w)
      if (piv_better(red_m[w], red_r[w], pmag, p)) { pmag = red_m[w]; p = red_r[w]; }
    const bool own_j = (j >= r0 && j < r0 + rc);
    if (COOP) {
      const int slot = jj & 1;
      if (tid == 0) { pm[slot * G + g] = pmag; pr[slot * G + g] = p; }
      const int lr = p - r0;
      for (int c = tid; c < nb; c += nth) {
        if (pmag >= 0.0 && lr >= 0 && lr < rc) pv[((size_t)slot * (G + 1) + g) * nb + c] = Ps[lr + (size_t)c * ch];
        if (own_j) pv[((size_t)slot * (G + 1) + G) * nb + c] = Ps[(j - r0) + (size_t)c * ch];
      }
      if (!group_barrier(bar, G, dev_err)) return;
      // the global pivot: warp 0 reduces the G published candidates (loads
      // bypass L1: the values were written by other CTAs)
      if (wid == 0) {
        double bm = -1.0;
        int brr = 0x7fffffff, bg = 0;
        for (int q2 = lane; q2 < G; q2 += 32) {
          const double m = __ldcg(&pm[slot * G + q2]);
          const int rr = __ldcg(&pr[slot * G + q2]);
          if (piv_better(m, rr, bm, brr)) { bm = m; brr = rr; bg = q2; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const double m2 = __shfl_down_sync(0xffffffffu, bm, o);
          const int r2 = __shfl_down_sync(0xffffffffu, brr, o);
          const int g2 = __shfl_down_sync(0xffffffffu, bg, o);
          if (piv_better(m2, r2, bm, brr)) { bm = m2; brr = r2; bg = g2; }
        }
        if (lane == 0) { red_m[0] = bm; red_r[0] = brr; s_bg = bg; }
      }
      __syncthreads();
      pmag = red_m[0];
      p = red_r[0];
      const double* wsrc = reinterpret_cast<const double*>(pv + ((size_t)slot * (G + 1) + s_bg) * nb);
      const double* rsrc = reinterpret_cast<const double*>(pv + ((size_t)slot * (G + 1) + G) * nb);
      double* wdst = reinterpret_cast<double*>(Wv);
      double* rdst = reinterpret_cast<double*>(Rv);
      constexpr int DW = sizeof(T) / sizeof(double);
      for (int c = tid; c < nb * DW; c += nth) {
        wdst[c] = __ldcg(&wsrc[c]);
        rdst[c] = __ldcg(&rsrc[c]);
      }
      __syncthreads();
      for (int c = tid; c < nb; c += nth) {
        if (own_j) Ps[(j - r0) + (size_t)c * ch] = Wv[c];
        if (p != j && p >= r0 && p < r0 + rc) Ps[(p - r0) + (size_t)c * ch] = Rv[c];
        if (c == jj) *reinterpret_cast<T*>(s_inv_raw) = (pmag == 0.0) ? T(0.0) : recip(Wv[c]);
      }
    } else {
      // one column per thread: read both rows, then write them swapped
      for (int c = tid; c < nb; c += nth) {
        const T wv = Ps[(p - r0) + (size_t)c * ch];
        const T rv = Ps[(j - r0) + (size_t)c * ch];
        Wv[c] = wv;
        Ps[(j - r0) + (size_t)c * ch] = wv;
        if (p != j) Ps[(p - r0) + (size_t)c * ch] = rv;
        if (c == jj) *reinterpret_cast<T*>(s_inv_raw) = (pmag == 0.0) ? T(0.0) : recip(wv);
      }
    }
    if (g == 0 && tid == 0) {
      ipiv[(int64_t)b * n + j] = p;
      if (pmag == 0.0 && info[b] == 0) info[b] = j + 1;
    }
    __syncthreads();
    // multipliers of this thread's rows (at most ch / RT + 1 of them are
    // kept: the rows rlo + rt, rlo + rt + RT, ...), then the update of its
    // columns; the next column's candidates are tracked by column lane 0
    const T inv = *reinterpret_cast<const T*>(s_inv_raw);
    const int rlo = max(0, j + 1 - r0);
    best = -1.0;
    brow = 0x7fffffff;
    if (CT == 1) {
      for (int r = rlo + rt; r < rc; r += RT) {
        const T l = Ps[r + (size_t)jj * ch] * inv;
        Ps[r + (size_t)jj * ch] = l;
        for (int c = jj + 1; c < nb; ++c) {
          const T v = fmsc(Ps[r + (size_t)c * ch], l, Wv[c]);
          Ps[r + (size_t)c * ch] = v;
          if (c == jj + 1) {
            const double m = mag1(v);
            if (piv_better(m, r0 + r, best, brow)) { best = m; brow = r0 + r; }
          }
        }
      }
    } else {
      // rc <= RT here: each thread has at most one row
      const int r = rlo + rt;
      T l = T(0.0);
      if (r < rc) l = Ps[r + (size_t)jj * ch] * inv;
      __syncthreads();
      if (r < rc) {
        if (ct == 0) Ps[r + (size_t)jj * ch] = l;
        for (int c = jj + 1 + ct; c < nb; c += CT) {
          const T v = fmsc(Ps[r + (size_t)c * ch], l, Wv[c]);
          Ps[r + (size_t)c * ch] = v;
          if (c == jj + 1) {
            const double m = mag1(v);
            if (piv_better(m, r0 + r, best, brow)) { best = m; brow = r0 + r; }
          }
        }
      }
    }
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c)
    for (int r = tid; r < rc; r += nth) Ab[(int64_t)(r0 + r) + (int64_t)(k0 + c) * lda] = Ps[r + (size_t)c * ch];
}

// Panel LU of tall panels in the distributed shared memory of a thread-block
// cluster.  The rows [k0, n) are split into CS contiguous chunks, one per CTA
// of the matrix's cluster, each held in that CTA's shared memory for the
// whole panel.  Rows never move during the panel: a chosen pivot row is only
// marked done, and the interchanges are recorded in LAPACK's form (ipiv) by
// a replay of the swap sequence on the panel's top positions (every warp
// keeps its own copy in registers, lane t for position k0 + t); at the end
// every row is written to its final position.
//
// Per column, one block barrier and one cluster barrier, and no remote load:
// every warp reduces its rows' candidates with shuffles; warp 0 reduces the
// eight warp candidates to the CTA's candidate (largest magnitude, and on ties
// the lowest current position -- the row order after the interchanges so far,
// which is LAPACK's choice), forms the reciprocal of its pivot-column entry
// and pushes the candidate -- magnitude, position, row, reciprocal and the
// row's panel values -- into the shared memory of every CTA of the cluster.
// After the cluster barrier every warp picks the same pivot from its own
// shared memory and updates its rows.  Candidates are double-buffered by
// column parity: a CTA pushes into a slot again only two columns later, after
// a barrier that every CTA reaches only once it has finished with the slot.
template <typename T>
__global__ void __launch_bounds__(256) k_lu_panel_cluster(BOp<T> A, int n, int k0, int nb, int* ipiv,
                                                          int* info) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int g = (int)cl.block_rank();
  const int b = blockIdx.x / CS;
  const int rows = n - k0;
  const int ch = (rows + CS - 1) / CS;
  const int r0 = k0 + g * ch;
  const int rc = max(0, min(ch, n - r0));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ps = reinterpret_cast<T*>(smem_raw);              // ch x nb, column-major
  T* cv = Ps + (size_t)ch * nb;                        // [2 slots][CS][nb]: every CTA's candidate row
  int* chosen = reinterpret_cast<int*>(cv + (size_t)2 * CS * nb);  // ch: pivot step of a row, or -1
  __shared__ long long wm[8];                          // warp candidates of this CTA
  __shared__ int wq[8], wp[8];
  __shared__ long long cm[2 * 16];                     // [slot][CTA] pushed candidates
  __shared__ int cq[2 * 16], cr[2 * 16];
  __shared__ double cinv_raw[2 * 16 * 2];              // their reciprocals (T)
  T* cinv = reinterpret_cast<T*>(cinv_raw);
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  const int kmax = (ch + nth - 1) / nth;               // row slots per thread, uniform over the CTA
  T* Ab = A.item(b);
  const int lda = A.ld;

  load_panel(Ps, Ab, lda, r0, k0, rc, ch, nb, tid, nth);
  for (int r = tid; r < ch; r += nth) chosen[r] = -1;
  int phys = k0 + lane;   // row now at position k0 + lane
  int pos = k0 + lane;    // current position of row k0 + lane
  // every CTA of the cluster has started before any writes into its shared memory
  cl.sync();
  // (magnitude, current position) orders candidates; prow is the row itself
  double best = -1.0;
  int bpos = 0x7fffffff, prow = -1;
  for (int r = tid; r < rc; r += nth) {
    const double m = mag1(Ps[r]);
    if (piv_better(m, r0 + r, best, bpos)) { best = m; bpos = r0 + r; prow = r0 + r; }
  }
  for (int jj = 0; jj < nb; ++jj) {
    const int slot = jj & 1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double m2 = __shfl_down_sync(0xffffffffu, best, o);
      const int q2 = __shfl_down_sync(0xffffffffu, bpos, o);
      const int p2 = __shfl_down_sync(0xffffffffu, prow, o);
      if (piv_better(m2, q2, best, bpos)) { best = m2; bpos = q2; prow = p2; }
    }
    if (lane == 0) { wm[wid] = __double_as_longlong(best); wq[wid] = bpos; wp[wid] = prow; }
    __syncthreads();
    if (wid == 0) {
      double m = -1.0;
      int q = 0x7fffffff, p = -1;
      if (lane < 8) { m = __longlong_as_double(wm[lane]); q = wq[lane]; p = wp[lane]; }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        const double m2 = __shfl_down_sync(0xffffffffu, m, o);
        const int q2 = __shfl_down_sync(0xffffffffu, q, o);
        const int p2 = __shfl_down_sync(0xffffffffu, p, o);
        if (piv_better(m2, q2, m, q)) { m = m2; q = q2; p = p2; }
      }
      m = __shfl_sync(0xffffffffu, m, 0);
      q = __shfl_sync(0xffffffffu, q, 0);
      p = __shfl_sync(0xffffffffu, p, 0);
      const bool has = m >= 0.0;
      const T v = (has && lane < nb) ? Ps[(p - r0) + (size_t)lane * ch] : T(0.0);
      T inv = T(0.0);
      if (lane == jj && has && m != 0.0) inv = recip(v);
      inv = shfl_val(inv, jj);
      for (int d = 0; d < CS; ++d)
        if (lane < nb) cl.map_shared_rank(cv, d)[((size_t)slot * CS + g) * nb + lane] = v;
      if (lane < CS) {
        const int e2 = slot * 16 + g;
        cl.map_shared_rank(cm, lane)[e2] = __double_as_longlong(m);
        cl.map_shared_rank(cq, lane)[e2] = q;
        cl.map_shared_rank(cr, lane)[e2] = p;
        cl.map_shared_rank(cinv, lane)[e2] = inv;
      }
    }
    cl.sync();
    // the pivot, chosen by every warp from its own CTA's shared memory
    double pm = -1.0;
    int pq = 0x7fffffff, pp = -1, pw = 0;
    if (lane < CS) {
      pm = __longlong_as_double(cm[slot * 16 + lane]);
      pq = cq[slot * 16 + lane];
      pp = cr[slot * 16 + lane];
      pw = lane;
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      const double m2 = __shfl_down_sync(0xffffffffu, pm, o);
      const int q2 = __shfl_down_sync(0xffffffffu, pq, o);
      const int p2 = __shfl_down_sync(0xffffffffu, pp, o);
      const int w2 = __shfl_down_sync(0xffffffffu, pw, o);
      if (piv_better(m2, q2, pm, pq)) { pm = m2; pq = q2; pp = p2; pw = w2; }
    }
    pm = __shfl_sync(0xffffffffu, pm, 0);
    pq = __shfl_sync(0xffffffffu, pq, 0);
    pp = __shfl_sync(0xffffffffu, pp, 0);
    pw = __shfl_sync(0xffffffffu, pw, 0);
    const T* Wv = cv + ((size_t)slot * CS + pw) * nb;
    const T inv = cinv[slot * 16 + pw];
    const int j = k0 + jj;
    if (pp >= r0 && pp < r0 + rc && (pp - r0) % nth == tid) chosen[pp - r0] = jj;
    // LAPACK interchange: position j <-> the winner's current position pq
    {
      const int rj = __shfl_sync(0xffffffffu, phys, jj);
      if (lane == rj - k0) pos = pq;
      if (pq - k0 < nb && lane == pq - k0) phys = rj;
      if (lane == jj) phys = pp;
      if (pp - k0 < nb && lane == pp - k0) pos = j;
    }
    if (g == 0 && tid == 0) {
      ipiv[(int64_t)b * n + j] = pq;
      if (pm == 0.0 && info[b] == 0) info[b] = j + 1;
    }
    best = -1.0;
    bpos = 0x7fffffff;
    prow = -1;
    for (int k = 0; k < kmax; ++k) {
      const int r = tid + k * nth;
      const int pr = r0 + r;
      const int ptop = __shfl_sync(0xffffffffu, pos, (pr - k0) & 31);
      if (r >= rc || chosen[r] >= 0) continue;
      const int cpos = pr - k0 < nb ? ptop : pr;  // after this column's interchange
      const T l = Ps[r + (size_t)jj * ch] * inv;
      Ps[r + (size_t)jj * ch] = l;
      for (int c = jj + 1; c < nb; ++c) {
        const T v = fmsc(Ps[r + (size_t)c * ch], l, Wv[c]);
        Ps[r + (size_t)c * ch] = v;
        if (c == jj + 1) {
          const double m = mag1(v);
          if (piv_better(m, cpos, best, bpos)) { best = m; bpos = cpos; prow = pr; }
        }
      }
    }
  }
  // rows to their final positions
  for (int k = 0; k < kmax; ++k) {
    const int r = tid + k * nth;
    const int pr = r0 + r;
    const int ptop = __shfl_sync(0xffffffffu, pos, (pr - k0) & 31);
    if (r >= rc) continue;
    int dst = pr;
    if (chosen[r] >= 0) dst = k0 + chosen[r];
    else if (pr - k0 < nb) dst = ptop;
    for (int c = 0; c < nb; ++c) Ab[(int64_t)dst + (int64_t)(k0 + c) * lda] = Ps[r + (size_t)c * ch];
  }
  cl.sync();
}

// Cluster shape for a panel of `rows` rows of `batch` matrices: a power of
// two of CTAs, at least 2, growing while a CTA would hold more than 128 rows
// and the clusters of all matrices still fit on the SMs at once (the panel's
// FP64 update is spread over more SMs), then until the chunk fits in shared
// memory; at most the largest cluster the device runs with the kernel's
// shared memory; 0 when the panel does not fit (the cooperative kernel is
// used then).
template <typename T>
size_t panel_cluster_smem(int rows, int nb, int cs) {
  const int ch = (rows + cs - 1) / cs;
  return ((size_t)ch * nb + 2 * (size_t)cs * nb) * sizeof(T) + (size_t)ch * sizeof(int) + 16;
}

template <typename T>
int panel_cluster_max() {
  static const int mx = [] {
    int dev = 0, smem_max = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_lu_panel_cluster<T>) != cudaSuccess ||
        cudaFuncSetAttribute(k_lu_panel_cluster<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_max - (int)fa.sharedSizeBytes) != cudaSuccess ||
        cudaFuncSetAttribute(k_lu_panel_cluster<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    // the largest cluster that can be resident with a near-full shared memory per CTA
    for (int cs = 16; cs >= 2; cs /= 2) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = (size_t)(smem_max - (int)fa.sharedSizeBytes);
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int ncl = 0;
      if (cudaOccupancyMaxActiveClusters(&ncl, (void*)k_lu_panel_cluster<T>, &cfg) == cudaSuccess && ncl > 0)
        return cs;
      cudaGetLastError();
    }
    return 0;
  }();
  return mx;
}

template <typename T>
int panel_cluster_size(int rows, int nb, int batch) {
  const int mx = panel_cluster_max<T>();
  if (mx < 2 || nb > 32) return 0;
  int smem_max = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int cs = 2;
  while (cs < mx && (rows + cs - 1) / cs > 128 && (int64_t)batch * cs * 2 <= device_sms()) cs *= 2;
  while (cs <= mx && panel_cluster_smem<T>(rows, nb, cs) + 8192 > (size_t)smem_max) cs *= 2;
  return cs <= mx ? cs : 0;
}

// Apply the panel's interchanges to every column outside the panel and
// solve U12 = L11^{-1} A12 for the columns in [k0 + nb, trsm_end).
//
// The nb interchanges are first composed into one permutation of at most
// 2 nb rows: warp 0 replays them with lane t holding the row now at
// position k0 + t, and for a step whose partner lies below the panel's top,
// lane jj recording that outside position and the row it received (a later
// step with the same partner takes the record over).  Every thread then reads
// all moved entries of its column at once and writes them back permuted --
// one round trip per column instead of one per interchange -- and solves its
// top block in registers.
template <typename T, int NB, bool REG>
__global__ void __launch_bounds__(128) k_laswp_trsm(BOp<T> A, int n, int k0, int nb, const int* ipiv,
                                                    int trsm_end) {
  extern __shared__ unsigned char smem_raw[];
  T* L11 = reinterpret_cast<T*>(smem_raw);  // nb x nb, column-major
  __shared__ int src_top[32], dst_out[32], src_out[32];
  const int b = blockIdx.y;
  T* Ab = A.item(b);
  const int lda = A.ld;
  const bool any_trsm = trsm_end > k0 + nb;
  if (any_trsm)
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      const int r = e % nb, c = e / nb;
      L11[e] = Ab[(int64_t)(k0 + r) + (int64_t)(k0 + c) * lda];
    }
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const int* ip = ipiv + (int64_t)b * n + k0;
    const int pl = lane < nb ? ip[lane] : 0;   // all interchanges in one load
    int content = k0 + lane;   // row whose entries sit at position k0 + lane
    int opos = -1, ocont = -1; // outside position last swapped at this lane's step, and its row
    for (int jj = 0; jj < nb; ++jj) {
      const int p = __shfl_sync(0xffffffffu, pl, jj);
      const int cj = __shfl_sync(0xffffffffu, content, jj);
      if (p < k0 + nb) {
        const int cp = __shfl_sync(0xffffffffu, content, p - k0);
        if (lane == jj) content = cp;
        if (lane == p - k0) content = cj;
      } else {
        const unsigned m = __ballot_sync(0xffffffffu, opos == p);
        const int owner = m ? 31 - __clz((int)m) : 0;
        const int held = __shfl_sync(0xffffffffu, ocont, owner);
        const int cur = m ? held : p;   // never swapped before: still row p
        if (m && lane == owner) opos = -1;
        if (lane == jj) { content = cur; opos = p; ocont = cj; }
      }
    }
    src_top[lane] = lane < nb ? content : 0;
    dst_out[lane] = lane < nb ? opos : -1;
    src_out[lane] = ocont;
  }
  __syncthreads();
  const int ncols_out = n - nb;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ncols_out; t += gridDim.x * blockDim.x) {
    const int c = (t < k0) ? t : t + nb;
    T* col = Ab + (int64_t)c * lda;
    T x[NB], xo[NB];
    if constexpr (REG) {
      // few CTAs (one or a few matrices): the whole column in registers,
      // every load in flight at once, the solve unrolled
#pragma unroll
      for (int q = 0; q < NB; ++q) {
        if (q < nb) x[q] = col[src_top[q]];
        if (q < nb && dst_out[q] >= 0) xo[q] = col[src_out[q]];
      }
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q < nb && dst_out[q] >= 0) col[dst_out[q]] = xo[q];
      if (c >= k0 + nb && c < trsm_end) {
#pragma unroll
        for (int jj = 1; jj < NB; ++jj) {
          if (jj < nb) {
            T s = x[jj];
#pragma unroll
            for (int ii = 0; ii < jj; ++ii) s = fmsc(s, L11[jj + ii * nb], x[ii]);
            x[jj] = s;
          }
        }
      }
#pragma unroll
      for (int q = 0; q < NB; ++q)
        if (q < nb) col[k0 + q] = x[q];
    } else {
      // many matrices: runtime-indexed arrays (local memory, L1-resident) keep
      // the registers, and so the occupancy that hides the FP64 solve's
      // latency, where the unrolled form would take ~250 registers a thread
      for (int q = 0; q < nb; ++q) {
        x[q] = col[src_top[q]];
        if (dst_out[q] >= 0) xo[q] = col[src_out[q]];
      }
      for (int q = 0; q < nb; ++q)
        if (dst_out[q] >= 0) col[dst_out[q]] = xo[q];
      if (c >= k0 + nb && c < trsm_end) {
        for (int jj = 1; jj < nb; ++jj) {
          T s = x[jj];
          for (int ii = 0; ii < jj; ++ii) s = fmsc(s, L11[jj + ii * nb], x[ii]);
          x[jj] = s;
        }
      }
#pragma unroll 8
      for (int q = 0; q < nb; ++q) col[k0 + q] = x[q];
    }
  }
}

__global__ void k_ipiv_to_perm(const int* ipiv, int* perm, int n, int batch) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const int* ip = ipiv + (int64_t)b * n;
  int* pm = perm + (int64_t)b * n;
  for (int i = 0; i < n; ++i) pm[i] = i;
  for (int j = 0; j < n; ++j) {
    int p = ip[j];
    if (p != j) { int t = pm[j]; pm[j] = pm[p]; pm[p] = t; }
  }
}

#include "tuned.h"

int& lu_tune(int param) {
  static int v[TUNE_COUNT] = {HPS_TUNED_LU_BASE_PANELS_FEW, HPS_TUNED_LU_BASE_PANELS_MANY,
                              HPS_TUNED_LU_FEW_MIN_N,       HPS_TUNED_LU_CLUSTER_PANEL,
                              HPS_TUNED_TC_MIN_WORK_REAL,   HPS_TUNED_TC_MIN_WORK_CPLX,
                              HPS_TUNED_TC_MIN_K,           HPS_TUNED_TC_CHUNK_MB,
                              HPS_TUNED_TC_PERSIST_MIN_K,   HPS_TUNED_LU_PANEL_NB_FEW};
  return v[param];
}

template <typename T> struct LuNB;
template <> struct LuNB<double> { enum { NB = 32 }; };
template <> struct LuNB<cplx> { enum { NB = 16 }; };

template <typename T>
int lu_group_size(int n, int batch, int num_sms) {
  const int nb = LuNB<T>::NB;
  // shared memory per CTA limited to ~96 KB for the panel chunk
  const size_t cap = 96 * 1024;
  int gmin = (int)((n * (size_t)nb * sizeof(T) + cap - 1) / cap);
  int G = std::max(1, gmin);
  // spread small batches over more CTAs so that all SMs get work
  int want = (2 * num_sms) / std::max(batch, 1);
  if (want > G) G = want;
  int gmax = std::max(1, n / 64);
  G = std::min(G, gmax);
  // cooperative residency: keep batch * G within one wave
  while (G > 1 && (int64_t)G * batch > 2 * num_sms) --G;
  return std::max(G, 1);
}

template <typename T>
size_t lu_pub_bytes(int n, int batch, int G) {
  if (G <= 1) return 0;
  const int nb = LuNB<T>::NB;
  size_t v = (size_t)batch * 2 * (G + 1) * nb * sizeof(T);
  size_t m = (size_t)batch * 2 * G * sizeof(double);
  size_t r = (size_t)batch * 2 * G * sizeof(int);
  return v + m + r + 256;
}

// Allow the panel kernel the device's whole opt-in shared memory once per
// process.  Setting the attribute per launch to the launch's own size would
// race between host threads that build concurrently (one thread's smaller
// value landing between another's set and launch).
template <typename T, bool COOP>
cudaError_t panel_smem_limit() {
  static const cudaError_t err = [] {
    int dev = 0, mx = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_lu_panel<T, COOP>);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_lu_panel<T, COOP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               mx - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) cudaGetLastError();
    return e;
  }();
  return err;
}

// Factor the panel A[k0:n, k0:k0+nb), apply its interchanges to every other
// column and solve U12 = L11^{-1} A12 for the columns [k0 + nb, trsm_end).
template <typename T>
static cudaError_t lu_leaf(BOp<T> A, int n, int k0, int nb, int trsm_end, int batch, int* ipiv, int* info,
                           unsigned* dev_err, int G, const LuWork& w, cudaStream_t st, Prof* pf) {
  constexpr double F = fma_flops<T>();
  const int nb0 = LuNB<T>::NB;
  cudaError_t e;
  const int rows = n - k0;
  int Gk = std::min(G, std::max(1, rows / 8));
  const int ch = (rows + Gk - 1) / Gk;
  size_t sm = ((size_t)ch * nb + 2 * nb) * sizeof(T);
  double pfl = 0.0;  // panel: rank-1 updates and multipliers (FMA-equivalents)
  for (int jj = 0; jj < nb; ++jj) {
    const double below = (double)(n - (k0 + jj) - 1);
    pfl += below * (nb - jj - 1) + below;
  }
  pfl *= F * batch;
  const int CS = (Gk > 1 && lu_tune(TUNE_LU_CLUSTER_PANEL)) ? panel_cluster_size<T>(rows, nb, batch) : 0;
  if (pf) {
    pf->begin(st);
    pf->note(rows, nb, CS > 1 ? CS : Gk, batch);  // k: CTAs per matrix
  }
  if (CS > 1) {
    // the panel in the distributed shared memory of a cluster per matrix
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(batch * CS);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = panel_cluster_smem<T>(rows, nb, CS);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_lu_panel_cluster<T>, A, n, k0, nb, ipiv, info);
    if (e != cudaSuccess) return e;
  } else if (Gk > 1) {
    T* pubv = reinterpret_cast<T*>(w.pub);
    double* pubm = reinterpret_cast<double*>(pubv + (size_t)batch * 2 * (G + 1) * nb0);
    int* pubr = reinterpret_cast<int*>(pubm + (size_t)batch * 2 * G);
    if ((e = panel_smem_limit<T, true>()) != cudaSuccess) return e;
    BOp<T> Aa = A;
    int nn = n, kk = k0, nbb = nb, GG = Gk;
    unsigned* bars = w.bars;
    void* args[] = {&Aa, &nn, &kk, &nbb, &GG, &ipiv, &info, &bars, &pubv, &pubm, &pubr, &dev_err};
    e = cudaLaunchCooperativeKernel((void*)k_lu_panel<T, true>, dim3(batch * Gk), dim3(256), args, sm, st);
    if (e != cudaSuccess) return e;
  } else {
    if ((e = panel_smem_limit<T, false>()) != cudaSuccess) return e;
    k_lu_panel<T, false><<<batch, 256, sm, st>>>(A, n, k0, nb, 1, ipiv, info, nullptr, nullptr, nullptr,
                                                 nullptr, dev_err);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (pf) pf->end(K_LU_PANEL, pfl, st);
  if (n > nb) {
    const int ncols = n - nb;
    // few matrices: 32-thread CTAs, so that the columns spread over the SMs
    const bool few = ((ncols + 127) / 128) * batch < 2 * device_sms();
    const int tpb = few ? 32 : 128;
    int bx = std::min((ncols + tpb - 1) / tpb, 1024);
    size_t sm2 = (size_t)nb * nb * sizeof(T);
    if (pf) {
      pf->begin(st);
      pf->note(nb, ncols, nb, batch);
    }
    if (few) k_laswp_trsm<T, LuNB<T>::NB, true><<<dim3(bx, batch), tpb, sm2, st>>>(A, n, k0, nb, ipiv, trsm_end);
    else k_laswp_trsm<T, LuNB<T>::NB, false><<<dim3(bx, batch), tpb, sm2, st>>>(A, n, k0, nb, ipiv, trsm_end);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (pf) pf->end(K_LASWP_TRSM, F * 0.5 * nb * (nb - 1) * (double)std::max(0, trsm_end - k0 - nb) * batch, st);
  }
  return cudaSuccess;
}

template <typename T>
static cudaError_t rtrsm_lower(BOp<T> LU, BOp<T> X, int p0, int n1, int nrhs, int batch, cudaStream_t st,
                               Prof* pf);

// Recursive LU with partial pivoting of the columns [c0, c1) (rows c0..n):
// factor the left half, U12 = L11^{-1} A12 by the recursive triangular
// solve, A22 -= A21 U12 as one product of inner dimension ~(c1 - c0) / 2,
// factor the right half.  Ranges of at most 4 panels are factored blocked
// right-looking (panel, interchanges + U12 within the range, update of the
// range's remaining columns), which keeps the launch count of the blocked
// algorithm; so are whole matrices when there are few of them (base_w = n).  The same pivots and operations as the blocked right-looking
// order; the bulk of the trailing updates becomes a few large-K products
// (on the tensor cores) instead of n / nb products of inner dimension nb.
template <typename T>
static cudaError_t rgetrf(BOp<T> A, int n, int c0, int c1, int base_w, int nb0, int batch, int* ipiv, int* info,
                          unsigned* dev_err, int G, const LuWork& w, cudaStream_t st, Prof* pf) {
  const int wdt = c1 - c0;
  cudaError_t e;
  if (wdt <= base_w) {
    for (int k0 = c0; k0 < c1; k0 += nb0) {
      const int nb = std::min(nb0, c1 - k0);
      if ((e = lu_leaf<T>(A, n, k0, nb, c1, batch, ipiv, info, dev_err, G, w, st, pf)) != cudaSuccess) return e;
      const int m2 = n - k0 - nb, n2 = c1 - k0 - nb;
      if (m2 > 0 && n2 > 0) {
        GemmArgs<T> g;
        g.M = m2; g.N = n2; g.K = nb; g.batch = batch;
        g.A = shifted(A, (int64_t)(k0 + nb) + (int64_t)k0 * A.ld);
        g.B = shifted(A, (int64_t)k0 + (int64_t)(k0 + nb) * A.ld);
        g.C = shifted(A, (int64_t)(k0 + nb) + (int64_t)(k0 + nb) * A.ld);
        g.alpha = T(-1.0); g.beta = T(1.0);
        if ((e = gemm(g, st, pf)) != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  }
  const int cm = c0 + ((wdt / 2 + nb0 - 1) / nb0) * nb0;
  if ((e = rgetrf<T>(A, n, c0, cm, base_w, nb0, batch, ipiv, info, dev_err, G, w, st, pf)) != cudaSuccess) return e;
  // U12: rows [c0, cm), columns [cm, c1)
  BOp<T> L11 = shifted(A, (int64_t)c0 + (int64_t)c0 * A.ld);
  BOp<T> A12 = shifted(A, (int64_t)c0 + (int64_t)cm * A.ld);
  if ((e = rtrsm_lower<T>(L11, A12, 0, cm - c0, c1 - cm, batch, st, pf)) != cudaSuccess) return e;
  if (n > cm) {
    GemmArgs<T> g;
    g.M = n - cm; g.N = c1 - cm; g.K = cm - c0; g.batch = batch;
    g.A = shifted(A, (int64_t)cm + (int64_t)c0 * A.ld);
    g.B = A12;
    g.C = shifted(A, (int64_t)cm + (int64_t)cm * A.ld);
    g.alpha = T(-1.0); g.beta = T(1.0);
    if ((e = gemm(g, st, pf)) != cudaSuccess) return e;
  }
  return rgetrf<T>(A, n, cm, c1, base_w, nb0, batch, ipiv, info, dev_err, G, w, st, pf);
}

template <typename T>
cudaError_t getrf(BOp<T> A, int n, int batch, int* ipiv, int* perm, int* info, unsigned* dev_err,
                  int G, const LuWork& w, cudaStream_t st, Prof* pf) {
  if (n <= 0 || batch <= 0) return cudaSuccess;
  cudaError_t e;
  // Few matrices: the recursion's triangular solves become many small
  // launches on a few SMs, so small orders keep the blocked right-looking
  // order (one fused interchange + U12 launch per panel); large ones recurse
  // so that the trailing updates are a few large-K products.
  const int nbp = LuNB<T>::NB;
  int base_w = lu_tune(TUNE_LU_BASE_PANELS_MANY) * nbp;
  // panel width: the kernels' maximum, or narrower for few matrices (the
  // panel's FP64 update, ~n^2 nb / 2 multiply-adds on the few SMs of a
  // cluster, against twice the panels and trailing updates of half the K)
  int pnb = nbp;
  if (batch < 8) {
    const int bp = lu_tune(TUNE_LU_BASE_PANELS_FEW);
    base_w = (bp <= 0 || n < lu_tune(TUNE_LU_FEW_MIN_N)) ? n : bp * nbp;
    pnb = std::max(8, std::min(nbp, lu_tune(TUNE_LU_PANEL_NB_FEW) / 8 * 8));
  }
  if (base_w < nbp) base_w = nbp;
  if ((e = rgetrf<T>(A, n, 0, n, base_w, pnb, batch, ipiv, info, dev_err, G, w, st, pf)) != cudaSuccess) return e;
  if (pf) pf->begin(st);
  k_ipiv_to_perm<<<(batch + 127) / 128, 128, 0, st>>>(ipiv, perm, n, batch);
  if (pf) pf->end(K_OTHER, 0.0, st);
  return cudaGetLastError();
}

// ------------------------------------------------------ triangular solve ----

template <typename T>
__global__ void k_permute_rows(BOp<T> src, BOp<T> dst, const int* perm, int n, int nrhs, int batch) {
  int64_t total = (int64_t)n * nrhs;
  for (int b = blockIdx.y; b < batch; b += gridDim.y) {
    const T* s = src.item(b);
    T* d = dst.item(b);
    const int* pm = perm + (int64_t)b * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
      int i = (int)(e % n), j = (int)(e / n);
      d[i + (int64_t)j * dst.ld] = s[pm[i] + (int64_t)j * src.ld];
    }
  }
}

template <typename T>
cudaError_t permute_rows(BOp<T> src, BOp<T> dst, const int* perm, int n, int nrhs, int batch,
                         cudaStream_t st, Prof* pf) {
  if (n <= 0 || nrhs <= 0 || batch <= 0) return cudaSuccess;
  int64_t total = (int64_t)n * nrhs;
  int bx = (int)std::min<int64_t>((total + 255) / 256, 2048);
  if (pf) pf->begin(st);
  k_permute_rows<T><<<dim3(bx, std::min(batch, 65535)), 256, 0, st>>>(src, dst, perm, n, nrhs, batch);
  if (pf) pf->end(K_GATHER, 0.0, st);
  return cudaGetLastError();
}

// Diagonal-block solve: X[p0:p0+pb, :] <- L[p0:p0+pb, p0:p0+pb]^{-1} X (unit
// lower, UPPER = false) or U^{-1} X (non-unit upper, UPPER = true).  One warp
// per right-hand side column, lane r owning row r (pb <= 32): each step
// broadcasts the solved entry with a shuffle and the lanes below (above)
// update their row, so a single column is solved in pb dependent steps.

template <typename T, bool UPPER>
__global__ void __launch_bounds__(128) k_trsm_diag(BOp<T> LU, BOp<T> X, int p0, int pb, int nrhs, int batch) {
  extern __shared__ unsigned char smem_raw[];
  T* Ls = reinterpret_cast<T*>(smem_raw);  // pb x pb, then pb reciprocals of the diagonal
  T* Dinv = Ls + pb * pb;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int b = blockIdx.y; b < batch; b += gridDim.y) {
    const T* Lb = LU.item(b);
    T* Xb = X.item(b);
    __syncthreads();
    for (int e = threadIdx.x; e < pb * pb; e += blockDim.x) {
      int r = e % pb, c = e / pb;
      Ls[e] = Lb[(int64_t)(p0 + r) + (int64_t)(p0 + c) * LU.ld];
    }
    __syncthreads();
    if (UPPER)
      for (int r = threadIdx.x; r < pb; r += blockDim.x) {
        const T d = Ls[r + r * pb];
        Dinv[r] = is_zero(d) ? T(0.0) : recip(d);
      }
    __syncthreads();
    for (int j = blockIdx.x * nw + wid; j < nrhs; j += gridDim.x * nw) {
      T* col = Xb + (int64_t)j * X.ld + p0;
      T x = lane < pb ? col[lane] : T(0.0);
      if (!UPPER) {
        for (int c = 0; c < pb - 1; ++c) {
          const T xc = shfl_val(x, c);
          if (lane > c && lane < pb) x = fmsc(x, Ls[lane + c * pb], xc);
        }
      } else {
        for (int c = pb - 1; c >= 0; --c) {
          if (lane == c) x = x * Dinv[c];
          const T xc = shfl_val(x, c);
          if (lane < c) x = fmsc(x, Ls[lane + c * pb], xc);
        }
      }
      if (lane < pb) col[lane] = x;
    }
  }
}

// Many right-hand sides: one thread per column, the block's pb x pb diagonal
// block staged once in shared memory for up to 128 columns.
template <typename T, bool UPPER>
__global__ void __launch_bounds__(128) k_trsm_diag_cols(BOp<T> LU, BOp<T> X, int p0, int pb, int nrhs, int batch) {
  extern __shared__ unsigned char smem_raw[];
  T* Ls = reinterpret_cast<T*>(smem_raw);
  T* Dinv = Ls + pb * pb;
  for (int b = blockIdx.y; b < batch; b += gridDim.y) {
    const T* Lb = LU.item(b);
    T* Xb = X.item(b);
    __syncthreads();
    for (int e = threadIdx.x; e < pb * pb; e += blockDim.x) {
      int r = e % pb, c = e / pb;
      Ls[e] = Lb[(int64_t)(p0 + r) + (int64_t)(p0 + c) * LU.ld];
    }
    __syncthreads();
    if (UPPER)
      for (int r = threadIdx.x; r < pb; r += blockDim.x) {
        const T d = Ls[r + r * pb];
        Dinv[r] = is_zero(d) ? T(0.0) : recip(d);
      }
    __syncthreads();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nrhs; j += gridDim.x * blockDim.x) {
      T* col = Xb + (int64_t)j * X.ld + p0;
      T x[32];
      for (int r = 0; r < pb; ++r) x[r] = col[r];
      if (!UPPER) {
        for (int r = 1; r < pb; ++r) {
          T s = x[r];
          for (int c = 0; c < r; ++c) s = fmsc(s, Ls[r + c * pb], x[c]);
          x[r] = s;
        }
      } else {
        for (int r = pb - 1; r >= 0; --r) {
          T s = x[r];
          for (int c = r + 1; c < pb; ++c) s = fmsc(s, Ls[r + c * pb], x[c]);
          x[r] = s * Dinv[r];
        }
      }
      for (int r = 0; r < pb; ++r) col[r] = x[r];
    }
  }
}

// Full 32-row diagonal blocks: a CTA takes CT right-hand sides of one
// matrix, loads the 32 x CT tile of X coalesced (a warp per column) into
// shared memory (stride 33: conflict-free per-thread columns), solves one
// column per thread in registers (fully unrolled), and stores coalesced.
template <typename T, bool UPPER, int CT>
__global__ void __launch_bounds__(CT) k_trsm32(BOp<T> LU, BOp<T> X, int p0, int nrhs, int batch) {
  __shared__ T Ls[32 * 32];
  __shared__ T Dinv[32];
  __shared__ T Xs[CT * 33];
  const int b = blockIdx.y;
  const T* Lb = LU.item(b);
  T* Xb = X.item(b);
  const int j0 = blockIdx.x * CT;
  const int ncol = min(CT, nrhs - j0);
  for (int e = threadIdx.x; e < 32 * 32; e += CT) {
    const int r = e & 31, c = e >> 5;
    Ls[e] = Lb[(int64_t)(p0 + r) + (int64_t)(p0 + c) * LU.ld];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = wid; c < ncol; c += CT / 32) Xs[c * 33 + lane] = Xb[(int64_t)(j0 + c) * X.ld + p0 + lane];
  __syncthreads();
  if (UPPER && threadIdx.x < 32) {
    const T d = Ls[threadIdx.x * 33];
    Dinv[threadIdx.x] = is_zero(d) ? T(0.0) : recip(d);
  }
  __syncthreads();
  if (threadIdx.x < ncol) {
    T x[32];
    T* xc = Xs + threadIdx.x * 33;
#pragma unroll
    for (int r = 0; r < 32; ++r) x[r] = xc[r];
    if (!UPPER) {
#pragma unroll
      for (int r = 1; r < 32; ++r) {
        T s2 = x[r];
#pragma unroll
        for (int c = 0; c < r; ++c) s2 = fmsc(s2, Ls[r + c * 32], x[c]);
        x[r] = s2;
      }
    } else {
#pragma unroll
      for (int r = 31; r >= 0; --r) {
        T s2 = x[r];
#pragma unroll
        for (int c = r + 1; c < 32; ++c) s2 = fmsc(s2, Ls[r + c * 32], x[c]);
        x[r] = s2 * Dinv[r];
      }
    }
#pragma unroll
    for (int r = 0; r < 32; ++r) xc[r] = x[r];
  }
  __syncthreads();
  for (int c = wid; c < ncol; c += CT / 32) Xb[(int64_t)(j0 + c) * X.ld + p0 + lane] = Xs[c * 33 + lane];
}

// Full 32-row diagonal blocks with few CTAs in the grid (few matrices):
// four threads per right-hand side, each holding 8 of the block's 32 rows.
// The row groups are solved in dependency order, each group's solution
// broadcast by shuffles to the four threads of its column, the later groups
// subtracting its contribution: the chain per column is four 8-row
// triangles and three 8 x 8 updates instead of one 32-row substitution, and
// the columns spread over four times the warps.
template <typename T, bool UPPER>
__global__ void __launch_bounds__(128) k_trsm32_g4(BOp<T> LU, BOp<T> X, int p0, int nrhs, int batch) {
  __shared__ T Ls[32 * 32];
  __shared__ T Dinv[32];
  __shared__ T Xs[32 * 33];
  const int b = blockIdx.y;
  const T* Lb = LU.item(b);
  T* Xb = X.item(b);
  const int j0 = blockIdx.x * 32;
  const int ncol = min(32, nrhs - j0);
  for (int e = threadIdx.x; e < 32 * 32; e += 128) {
    const int r = e & 31, c = e >> 5;
    Ls[e] = Lb[(int64_t)(p0 + r) + (int64_t)(p0 + c) * LU.ld];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = wid; c < ncol; c += 4) Xs[c * 33 + lane] = Xb[(int64_t)(j0 + c) * X.ld + p0 + lane];
  __syncthreads();
  if (UPPER && threadIdx.x < 32) {
    const T d = Ls[threadIdx.x * 33];
    Dinv[threadIdx.x] = is_zero(d) ? T(0.0) : recip(d);
  }
  __syncthreads();
  const int col = threadIdx.x >> 2, g = threadIdx.x & 3;
  const bool live = col < ncol;
  const int lane0 = lane & ~3;   // the column's first lane
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = live ? Xs[col * 33 + 8 * g + i] : T(0.0);
#pragma unroll
  for (int step = 0; step < 4; ++step) {
    const int blk = UPPER ? 3 - step : step;
    if (g == blk) {
      if (!UPPER) {
#pragma unroll
        for (int i = 1; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < i; ++j) x[i] = fmsc(x[i], Ls[(8 * g + i) + (8 * g + j) * 32], x[j]);
      } else {
#pragma unroll
        for (int i = 7; i >= 0; --i) {
          T sacc = x[i];
#pragma unroll
          for (int j = i + 1; j < 8; ++j) sacc = fmsc(sacc, Ls[(8 * g + i) + (8 * g + j) * 32], x[j]);
          x[i] = sacc * Dinv[8 * g + i];
        }
      }
    }
    T xb[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) xb[j] = shfl_val(x[j], lane0 | blk);
    if (UPPER ? g < blk : g > blk) {
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) x[i] = fmsc(x[i], Ls[(8 * g + i) + (8 * blk + j) * 32], xb[j]);
    }
  }
  if (live) {
#pragma unroll
    for (int i = 0; i < 8; ++i) Xs[col * 33 + 8 * g + i] = x[i];
  }
  __syncthreads();
  for (int c = wid; c < ncol; c += 4) Xb[(int64_t)(j0 + c) * X.ld + p0 + lane] = Xs[c * 33 + lane];
}

template <typename T, bool UPPER>
cudaError_t trsm_diag(BOp<T> LU, BOp<T> X, int p0, int pb, int nrhs, int batch, cudaStream_t st) {
  const size_t sm = ((size_t)pb * pb + pb) * sizeof(T);
  const int by = std::min(batch, 65535);
  if (pb == 32 && nrhs >= 16 && batch <= 65535) {
    // 128 columns per CTA (real data) unless that leaves most SMs idle; the
    // complex tile keeps 32 so that static shared memory stays below 48 KB;
    // a grid of at most one such CTA per SM splits each column over four
    // threads (shorter chains on more SMSPs; with more CTAs than SMs the
    // split form's extra instructions cost more than its latency saves:
    // measured on 1793 complex columns of 4 matrices, 4.6 -> 5.2 ms)
    const int ctas32 = ((nrhs + 31) / 32) * batch;
    bool wide = false;
    if constexpr (sizeof(T) == 8) {
      wide = ((nrhs + 127) / 128) * batch >= 2 * device_sms();
      if (wide) k_trsm32<T, UPPER, 128><<<dim3((nrhs + 127) / 128, batch), 128, 0, st>>>(LU, X, p0, nrhs, batch);
    }
    if (!wide) {
      if (ctas32 <= device_sms())
        k_trsm32_g4<T, UPPER><<<dim3((nrhs + 31) / 32, batch), 128, 0, st>>>(LU, X, p0, nrhs, batch);
      else
        k_trsm32<T, UPPER, 32><<<dim3((nrhs + 31) / 32, batch), 32, 0, st>>>(LU, X, p0, nrhs, batch);
    }
  } else if (nrhs >= 16) {
    const int bx = std::min((nrhs + 127) / 128, 1024);
    k_trsm_diag_cols<T, UPPER><<<dim3(bx, by), 128, sm, st>>>(LU, X, p0, pb, nrhs, batch);
  } else {
    const int bx = std::min((nrhs + 3) / 4, 1024);
    k_trsm_diag<T, UPPER><<<dim3(bx, by), 128, sm, st>>>(LU, X, p0, pb, nrhs, batch);
  }
  return cudaGetLastError();
}

// Recursive triangular solves on rows [p0, p0 + n1) of X: split at a
// multiple of 32 near the middle, solve the first half, update the second
// with one product of inner dimension ~n1/2, solve the second half; 32-row
// diagonal blocks at the leaves.  Same operations as the blocked
// right-looking order, but the updates are few large-K products (the bulk
// runs on the tensor cores) instead of n/32 products of inner dimension 32
// that each re-read the rest of X.
template <typename T>
static cudaError_t rtrsm_lower(BOp<T> LU, BOp<T> X, int p0, int n1, int nrhs, int batch, cudaStream_t st,
                               Prof* pf) {
  constexpr double F = fma_flops<T>();
  cudaError_t e;
  if (n1 <= 32) {
    if (pf) {
      pf->begin(st);
      pf->note(n1, nrhs, n1, batch);
    }
    if ((e = trsm_diag<T, false>(LU, X, p0, n1, nrhs, batch, st)) != cudaSuccess) return e;
    if (pf) pf->end(K_TRSM_DIAG, F * 0.5 * n1 * (n1 - 1) * (double)nrhs * batch, st);
    return cudaSuccess;
  }
  const int h = ((n1 / 2 + 31) / 32) * 32;
  if ((e = rtrsm_lower<T>(LU, X, p0, h, nrhs, batch, st, pf)) != cudaSuccess) return e;
  GemmArgs<T> g;
  g.M = n1 - h; g.N = nrhs; g.K = h; g.batch = batch;
  g.A = shifted(LU, (int64_t)(p0 + h) + (int64_t)p0 * LU.ld);
  g.B = shifted(X, (int64_t)p0);
  g.C = shifted(X, (int64_t)(p0 + h));
  g.alpha = T(-1.0); g.beta = T(1.0);
  if ((e = gemm(g, st, pf)) != cudaSuccess) return e;
  return rtrsm_lower<T>(LU, X, p0 + h, n1 - h, nrhs, batch, st, pf);
}

template <typename T>
static cudaError_t rtrsm_upper(BOp<T> LU, BOp<T> X, int p0, int n1, int nrhs, int batch, cudaStream_t st,
                               Prof* pf) {
  constexpr double F = fma_flops<T>();
  cudaError_t e;
  if (n1 <= 32) {
    if (pf) {
      pf->begin(st);
      pf->note(n1, nrhs, n1, batch);
    }
    if ((e = trsm_diag<T, true>(LU, X, p0, n1, nrhs, batch, st)) != cudaSuccess) return e;
    if (pf) pf->end(K_TRSM_DIAG, F * (0.5 * n1 * (n1 - 1) + n1) * (double)nrhs * batch, st);
    return cudaSuccess;
  }
  const int h = ((n1 / 2 + 31) / 32) * 32;
  if ((e = rtrsm_upper<T>(LU, X, p0 + h, n1 - h, nrhs, batch, st, pf)) != cudaSuccess) return e;
  GemmArgs<T> g;
  g.M = h; g.N = nrhs; g.K = n1 - h; g.batch = batch;
  g.A = shifted(LU, (int64_t)p0 + (int64_t)(p0 + h) * LU.ld);
  g.B = shifted(X, (int64_t)(p0 + h));
  g.C = shifted(X, (int64_t)p0);
  g.alpha = T(-1.0); g.beta = T(1.0);
  if ((e = gemm(g, st, pf)) != cudaSuccess) return e;
  return rtrsm_upper<T>(LU, X, p0, h, nrhs, batch, st, pf);
}

template <typename T>
cudaError_t getrs_inplace(BOp<T> LU, int n, BOp<T> X, int nrhs, int batch, cudaStream_t st,
                          Prof* pf) {
  if (n <= 0 || nrhs <= 0 || batch <= 0) return cudaSuccess;
  cudaError_t e;
  // forward: unit lower; backward: non-unit upper
  if ((e = rtrsm_lower<T>(LU, X, 0, n, nrhs, batch, st, pf)) != cudaSuccess) return e;
  return rtrsm_upper<T>(LU, X, 0, n, nrhs, batch, st, pf);
}

// --------------------------------------------- flag-ordered solve ----
//
// Triangular solve of a single large factor with few right-hand sides.  The
// blocked getrs issues two launches per 32 rows, each far too small to fill
// the GPU; here one launch per triangle walks the 32-row blocks in dependency
// order (forward: first to last; backward: last to first).  CTA c takes the
// logical blocks c, c + G, c + 2G, ... in increasing order.  For each, all
// eight warps subtract the contributions of the earlier blocks as their
// solutions are published, warp w taking columns 4w .. 4w + 3 of every
// earlier block (each warp loads its matrix entries before it waits, and the
// FP64 work of one 32 x 32 block is spread over the whole SM); the block's
// solution is then the product of the precomputed inverse of its 32 x 32
// diagonal block (k_diag_block_inv) with the reduced right-hand side, split
// the same way.  The launch is cooperative, so every CTA is resident, and the
// earliest unfinished block depends only on finished ones: the walk always
// makes progress.  Waits are bounded: on timeout the flag error word is set
// and the block proceeds (wrong values, but the launch ends).
template <typename T, int NR, bool UPPER>
__global__ void __launch_bounds__(256) k_trsv_flags(const T* __restrict__ LU, int ld, int n, T* X, int ldx,
                                                   int nrhs, const T* __restrict__ dinv, unsigned* flags,
                                                   unsigned epoch, volatile int* err) {
  __shared__ T part[8][NR][32];
  __shared__ T y[NR][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nblk = (n + 31) / 32;
  for (int t = blockIdx.x; t < nblk; t += gridDim.x) {
    const int j = UPPER ? nblk - 1 - t : t;
    const int r = j * 32 + lane;
    const bool rv = r < n;
    T acc[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = T(0.0);
    for (int tp = 0; tp < t; ++tp) {
      const int i = UPPER ? nblk - 1 - tp : tp;
      const int qn = min(32, n - i * 32);
      T a[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int q = 4 * w + k;
        a[k] = (rv && q < qn) ? LU[(int64_t)r + (int64_t)(i * 32 + q) * ld] : T(0.0);
      }
      if (lane == 0) {
        if (!wait_flag(flags + i, epoch, 1ull << 24)) *err = 1;
        __threadfence();
      }
      __syncwarp();
      T xi[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        const int q = 4 * w + lane;
        xi[c] = (lane < 4 && q < qn && c < nrhs) ? ld_cg(X + (int64_t)(i * 32 + q) + (int64_t)c * ldx) : T(0.0);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = fmsc(acc[c], a[k], shfl_val(xi[c], k));
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) part[w][c][lane] = acc[c];
    __syncthreads();
    if (w == 0) {
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        T sum = (rv && c < nrhs) ? X[r + (int64_t)c * ldx] : T(0.0);
        for (int k = 0; k < 8; ++k) sum = sum + part[k][c][lane];
        y[c][lane] = sum;
      }
    }
    __syncthreads();
    // x_j = inv(diagonal block j) y, the inverse column-major 32 x 32
    const T* Dj = dinv + (int64_t)j * 1024;
    T acc2[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc2[c] = T(0.0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = 4 * w + k;
      const T dq = Dj[lane + 32 * q];
#pragma unroll
      for (int c = 0; c < NR; ++c) acc2[c] = fmac(acc2[c], dq, y[c][q]);
    }
#pragma unroll
    for (int c = 0; c < NR; ++c) part[w][c][lane] = acc2[c];
    __syncthreads();
    if (w == 0) {
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        T xs = T(0.0);
        for (int k = 0; k < 8; ++k) xs = xs + part[k][c][lane];
        if (rv && c < nrhs) X[r + (int64_t)c * ldx] = xs;
      }
      __threadfence();
      __syncwarp();
      if (lane == 0) atomicExch(flags + j, epoch);
    }
    __syncthreads();
  }
}

// Inverses of the 32 x 32 diagonal blocks of an LU factor (column-major,
// 32 x 32 each): tri 0 the unit lower L_jj, tri 1 the upper U_jj; a partial
// last block is completed with the identity, a zero pivot gives a zero row
// of the inverse (a singular factor was reported by the factorisation).
// One CTA per (block, triangle), thread c computes column c by substitution.
template <typename T>
__global__ void __launch_bounds__(32) k_diag_block_inv(const T* __restrict__ LU, int ld, int n, T* out) {
  const int j = blockIdx.x, tri = blockIdx.y, c = threadIdx.x, nblk = gridDim.x;
  const int pb = min(32, n - j * 32);
  const T* Dj = LU + (int64_t)(j * 32) + (int64_t)(j * 32) * ld;
  T x[32];
  if (tri == 0) {
#pragma unroll
    for (int rr = 0; rr < 32; ++rr) {
      T v = rr == c ? T(1.0) : T(0.0);
      if (rr < pb)
        for (int k = 0; k < rr; ++k) v = fmsc(v, Dj[rr + (int64_t)k * ld], x[k]);
      x[rr] = v;
    }
  } else {
#pragma unroll
    for (int rr = 31; rr >= 0; --rr) {
      T v = rr == c ? T(1.0) : T(0.0);
      if (rr < pb) {
        for (int k = rr + 1; k < pb; ++k) v = fmsc(v, Dj[rr + (int64_t)k * ld], x[k]);
        const T d = Dj[rr + (int64_t)rr * ld];
        v = is_zero(d) ? T(0.0) : v * recip(d);
      }
      x[rr] = v;
    }
  }
  T* o = out + ((int64_t)tri * nblk + j) * 1024;
#pragma unroll
  for (int rr = 0; rr < 32; ++rr) o[rr + 32 * c] = x[rr];
}

template <typename T>
bool trsv_flags_applicable(int n, int nrhs, int batch, const TrsvWork& w) {
  return batch == 1 && nrhs >= 1 && nrhs <= 8 && n >= 128 && w.flags && w.dev_err && w.dinv &&
         (n + 31) / 32 <= w.nflags;
}

template <typename T, int NR, bool UPPER>
cudaError_t launch_trsv_flags(const T* LU, int n, int ld, T* X, int ldx, int nrhs, TrsvWork& w,
                              cudaStream_t st) {
  // resident CTAs of this kernel on the whole GPU (thread-safe one-time
  // initialisation; 0 if the query failed)
  static const int resident = [] {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trsv_flags<T, NR, UPPER>, 256, 0) !=
            cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return per_sm * sms;
  }();
  if (resident <= 0) return cudaErrorInvalidConfiguration;
  const int nblk = (n + 31) / 32;
  const int G = std::max(1, std::min(nblk, resident));
  const unsigned ep = ++w.epoch;
  unsigned* fl = w.flags;
  int* errp = const_cast<int*>(w.dev_err);
  const T* dv = static_cast<const T*>(w.dinv) + (UPPER ? (int64_t)nblk * 1024 : 0);
  void* args[] = {(void*)&LU, &ld, &n, &X, &ldx, &nrhs, (void*)&dv, &fl, (void*)&ep, &errp};
  return cudaLaunchCooperativeKernel((void*)k_trsv_flags<T, NR, UPPER>, dim3(G), dim3(256), args, 0, st);
}

template <typename T, bool UPPER>
cudaError_t trsv_flags_dispatch(const T* LU, int n, int ld, T* X, int ldx, int nrhs, TrsvWork& w,
                                cudaStream_t st) {
  if (nrhs == 1) return launch_trsv_flags<T, 1, UPPER>(LU, n, ld, X, ldx, nrhs, w, st);
  if (nrhs == 2) return launch_trsv_flags<T, 2, UPPER>(LU, n, ld, X, ldx, nrhs, w, st);
  if (nrhs <= 4) return launch_trsv_flags<T, 4, UPPER>(LU, n, ld, X, ldx, nrhs, w, st);
  return launch_trsv_flags<T, 8, UPPER>(LU, n, ld, X, ldx, nrhs, w, st);
}

template <typename T>
cudaError_t getrs_flags(const T* LU, int n, int ld, T* X, int ldx, int nrhs, TrsvWork& w, cudaStream_t st,
                        Prof* pf) {
  constexpr double F = fma_flops<T>();
  cudaError_t e;
  if (!w.dinv_ready) {
    // the diagonal blocks' inverses, once per factor (its storage was sized
    // with the flags)
    if (pf) pf->begin(st);
    k_diag_block_inv<T><<<dim3((n + 31) / 32, 2), 32, 0, st>>>(LU, ld, n, static_cast<T*>(w.dinv));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (pf) pf->end(K_OTHER, 0.0, st);
    w.dinv_ready = true;
  }
  if (pf) {
    pf->begin(st);
    pf->note(n, nrhs, 32, 1);
  }
  if ((e = trsv_flags_dispatch<T, false>(LU, n, ld, X, ldx, nrhs, w, st)) != cudaSuccess) return e;
  if (pf) pf->end(K_TRSM_DIAG, F * 0.5 * n * (double)(n - 1) * nrhs, st);
  if (pf) {
    pf->begin(st);
    pf->note(n, nrhs, 32, 1);
  }
  if ((e = trsv_flags_dispatch<T, true>(LU, n, ld, X, ldx, nrhs, w, st)) != cudaSuccess) return e;
  if (pf) pf->end(K_TRSM_DIAG, F * (0.5 * n * (double)(n - 1) + n) * nrhs, st);
  return cudaSuccess;
}

// ------------------------------------------------- conjugate transposes ----

namespace {
inline int grid_n(int64_t total, int threads = 256) {
  int64_t b = (total + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 65535 * 8));
}
}  // namespace

// dst(perm[i], j) = src(i, j): the inverse of permute_rows.
template <typename T>
__global__ void k_permute_rows_inv(BOp<T> src, BOp<T> dst, const int* perm, int n, int nrhs, int batch) {
  const int64_t per = (int64_t)n * nrhs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * batch; e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / per);
    const int rc = (int)(e % per);
    const int i = rc % n, j = rc / n;
    dst.item(b)[perm[(int64_t)b * n + i] + (int64_t)j * dst.ld] = src.item(b)[i + (int64_t)j * src.ld];
  }
}

// Diagonal-block solves with the conjugate transposes of the LU factors:
// LOWER: U^H w = y (U^H is lower triangular); else L^H z = w (upper, unit).
template <typename T, bool LOWER>
__global__ void k_trsm_diag_h(BOp<T> LU, BOp<T> X, int p0, int pb, int nrhs, int batch) {
  for (int b = blockIdx.y; b < batch; b += gridDim.y) {
    const T* Lb = LU.item(b);
    T* Xb = X.item(b);
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nrhs; j += gridDim.x * blockDim.x) {
      T* col = Xb + (int64_t)j * X.ld + p0;
      if (LOWER) {
        for (int r = 0; r < pb; ++r) {
          T s = col[r];
          for (int c = 0; c < r; ++c) s = fmsc(s, conj_of(Lb[(int64_t)(p0 + c) + (int64_t)(p0 + r) * LU.ld]), col[c]);
          const T d = conj_of(Lb[(int64_t)(p0 + r) + (int64_t)(p0 + r) * LU.ld]);
          col[r] = is_zero(d) ? T(0.0) : s * recip(d);
        }
      } else {
        for (int r = pb - 1; r >= 0; --r) {
          T s = col[r];
          for (int c = r + 1; c < pb; ++c)
            s = fmsc(s, conj_of(Lb[(int64_t)(p0 + c) + (int64_t)(p0 + r) * LU.ld]), col[c]);
          col[r] = s;
        }
      }
    }
  }
}

template <typename T>
cudaError_t permute_rows_inv(BOp<T> src, BOp<T> dst, const int* perm, int n, int nrhs, int batch, cudaStream_t st) {
  k_permute_rows_inv<T><<<grid_n((int64_t)n * nrhs * batch), 256, 0, st>>>(src, dst, perm, n, nrhs, batch);
  return cudaGetLastError();
}

// X <- (U^H)^{-1} then (L^H)^{-1}: the conjugate transpose of getrs_inplace
// (without the row permutation, which the caller applies after).
template <typename T>
cudaError_t getrs_h(BOp<T> LU, int n, BOp<T> X, int nrhs, int batch, cudaStream_t st, Prof* pf) {
  const int pb0 = 32;
  const int by = std::min(batch, 65535);
  const int bx = std::min((nrhs + 127) / 128, 1024);
  cudaError_t e;
  for (int p0 = 0; p0 < n; p0 += pb0) {
    const int pb = std::min(pb0, n - p0);
    k_trsm_diag_h<T, true><<<dim3(bx, by), 128, 0, st>>>(LU, X, p0, pb, nrhs, batch);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int rest = n - p0 - pb;
    if (rest > 0) {
      GemmArgs<T> g;
      g.M = rest; g.N = nrhs; g.K = pb; g.batch = batch;
      g.A = shifted(LU, (int64_t)p0 + (int64_t)(p0 + pb) * LU.ld);  // U(p0 .., p0 + pb ..)
      g.ta = true;
      g.B = shifted(X, (int64_t)p0);
      g.C = shifted(X, (int64_t)(p0 + pb));
      g.alpha = T(-1.0); g.beta = T(1.0);
      if ((e = gemm<T>(g, st, pf)) != cudaSuccess) return e;
    }
  }
  const int npan = (n + pb0 - 1) / pb0;
  for (int pi = npan - 1; pi >= 0; --pi) {
    const int p0 = pi * pb0, pb = std::min(pb0, n - p0);
    k_trsm_diag_h<T, false><<<dim3(bx, by), 128, 0, st>>>(LU, X, p0, pb, nrhs, batch);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (p0 > 0) {
      GemmArgs<T> g;
      g.M = p0; g.N = nrhs; g.K = pb; g.batch = batch;
      g.A = shifted(LU, (int64_t)p0);  // L(p0 .., 0 ..)
      g.ta = true;
      g.B = shifted(X, (int64_t)p0);
      g.C = X;
      g.alpha = T(-1.0); g.beta = T(1.0);
      if ((e = gemm<T>(g, st, pf)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// ------------------------------------------------------- instantiation ----

#define HPS_INST(T)                                                                              \
  template cudaError_t gemm<T>(const GemmArgs<T>&, cudaStream_t, Prof*);                         \
  template cudaError_t fill<T>(BOp<T>, int, int, int, T, T, cudaStream_t, Prof*);                \
  template int lu_group_size<T>(int, int, int);                                                  \
  template size_t lu_pub_bytes<T>(int, int, int);                                                \
  template cudaError_t getrf<T>(BOp<T>, int, int, int*, int*, int*, unsigned*, int,              \
                                const LuWork&, cudaStream_t, Prof*);                             \
  template cudaError_t permute_rows<T>(BOp<T>, BOp<T>, const int*, int, int, int, cudaStream_t,  \
                                       Prof*);                                                   \
  template cudaError_t getrs_inplace<T>(BOp<T>, int, BOp<T>, int, int, cudaStream_t, Prof*);                   \
  template bool trsv_flags_applicable<T>(int, int, int, const TrsvWork&);                        \
  template cudaError_t getrs_flags<T>(const T*, int, int, T*, int, int, TrsvWork&, cudaStream_t, Prof*); \
  template cudaError_t permute_rows_inv<T>(BOp<T>, BOp<T>, const int*, int, int, int, cudaStream_t);    \
  template cudaError_t getrs_h<T>(BOp<T>, int, BOp<T>, int, int, cudaStream_t, Prof*);

HPS_INST(double)
HPS_INST(cplx)


// ----------------------------------------------------------------------------
// Bounded-wait check (hps_debug_wait_timeout): one CTA runs one of the
// library's bounded waits on a word that nothing else writes.  which 0: the
// inter-CTA group barrier with a group of two CTAs of which only this one
// arrives (satisfied: a group of one); which 1: the flag wait of the
// flag-ordered triangular solves on a flag nothing sets (satisfied: the flag
// already holds the awaited value).  A wait that gives up sets
// DEV_ERR_TIMEOUT in *err.
__global__ void k_debug_wait(int which, int satisfied, unsigned* words, unsigned long long limit, unsigned* err) {
  if (which == 0) {
    group_barrier(words, satisfied ? 1u : 2u, err, limit);
  } else if (threadIdx.x == 0) {
    if (satisfied) words[2] = 7u;
    __threadfence();
    if (!wait_flag(words + 2, 7u, limit)) atomicOr(err, DEV_ERR_TIMEOUT);
  }
}

cudaError_t debug_wait(int which, int satisfied, unsigned* words, unsigned long long limit, unsigned* err,
                       cudaStream_t st) {
  k_debug_wait<<<1, 128, 0, st>>>(which, satisfied, words, limit, err);
  return cudaGetLastError();
}

}  // namespace hps
