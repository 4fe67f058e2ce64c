// FP64 and complex128 GEMMs on the tcgen05 tensor cores by exact digit
// slicing (an Ozaki-type splitting of each operand into bf16 digit matrices).
//
// Why: the FP64 FMA pipe of this GPU does 4 flop/clk/SM, while the bf16
// tensor cores do ~7000.  A real product C = A B is computed as
//
//   A(i, k) ~ 2^{e_i} sum_p a_p(i, k) 2^{-6p},   B(k, j) ~ 2^{f_j} sum_q b_q(k, j) 2^{-6q},
//
// p, q = 1..10, where 2^{e_i} (2^{f_j}) is the power of two above the
// largest |A(i, :)| (|B(:, j)|) and the digits are the balanced base-64
// digits of the scaled value rounded to 60 fraction bits: the leading digit
// in [-64, 64], the others in [-32, 31].  Integers of that size are exact in
// bf16, their products are exact in the fp32 accumulators of tcgen05.mma, and
// so are sums of up to 2^22 / 12288 of the products that share one
// anti-diagonal d = p + q (weight 2^{-6d}).  The product keeps the pairs with
// p + q <= 11 and accumulates each diagonal exactly in its own TMEM
// accumulator over K chunks of up to 256.  The epilogue converts the ten
// diagonal sums to integers, adds them in a 64-bit fixed-point integer (the
// low diagonals first at full precision, then rounded once) and scales by
// 2^{e_i + f_j} into FP64.  Errors: operand rounding 2^{-61} 2^{e_i} per
// entry (unbiased), dropped pairs about 2^{-59} K 2^{e_i + f_j}, half a unit
// of the fixed point (2^{-lsb}, lsb = 62 - ceil(log2 K)) per chunk, and the
// final rounding to FP64: at or below FP64's own rounding error for a dot
// product of length K when rows and columns are not far from their largest
// entries.
//
// Layout: the slicing kernel writes each operand's digits, K-major, in the
// tensor core's canonical no-swizzle layout (8-row x 16-byte core matrices;
// a 16-deep k step of a 128-row A tile is one 4 KB block per digit, of a
// 48-column B tile one 1.5 KB block), so that one k step of all digits is one
// contiguous bulk copy (cp.async.bulk) per operand.  The GEMM kernel computes
// 128 x 48 output tiles, one CTA per SM walking the launch's tiles: a
// producer warp streams the digit blocks through a 3-stage shared-memory
// ring, one thread issues the products as 15 MMAs per k step (digits of B
// stacked along N, up to 5 per MMA, land in adjacent diagonal accumulators),
// ten TMEM accumulators take 480 of the 512 columns, and eight epilogue
// warps (two per TMEM lane quarter, one per half of the columns) read them
// back while the next tile's copies and products proceed.  A product with
// few rows may run transposed (C^T = B^T A^T, C's rows on the 48-wide side).
//
// Complex products are two launches, one per component of C, each
// accumulating two real products in the same TMEM accumulators
// (Re = Ar Br - Ai Bi with the second product negated by the MMA's negate-B
// bit, Im = Ar Bi + Ai Br): the real and imaginary parts of a row of A (a
// column of B) are scaled by one power of two, above the largest |re| or |im|
// of the row, so that their digit products carry the same weights; the
// error bound above then holds with 2K terms and those joint row scales.
#include "devmem.h"
#include "linalg.h"

#include <algorithm>
#include <mutex>
#include <type_traits>

namespace hps {
namespace tc {

constexpr int DIG = 10;             // digits per operand
constexpr int BITS = 6;             // bits per digit
constexpr int FRAC = DIG * BITS;    // fraction bits of the scaled operands
constexpr int DSUM = 11;            // keep digit pairs with p + q <= DSUM (1-based)
constexpr int NDIAG = DSUM - 1;     // accumulators: d = 2 .. DSUM
constexpr int TM = 128, TN = 48, TK = 16;
constexpr int KC = 256;             // k per exact fp32 accumulation chunk
constexpr int KCT = KC / TK;        // k steps per chunk
constexpr int ABLK = TM * TK * 2;   // bytes of one digit of an A tile k step
constexpr int BBLK = TN * TK * 2;
constexpr int ASTG = DIG * ABLK;
constexpr int BSTG = DIG * BBLK;
constexpr int STAGE = ASTG + BSTG;
constexpr int QGRP = 5;             // B digits stacked into one MMA (N = 5 * 48 = 240 <= 256)
constexpr int NST = 3;
constexpr int TMP = TM + 1;          // C staging row stride (odd: transposed reads spread over banks)
constexpr int CSTG = TN * TMP * 8;    // the C tile staged for the epilogue (column-major)
constexpr int SMEM = NST * STAGE + CSTG;
constexpr int TMEM_COLS = 512;
constexpr int EPI_WARPS = 8;        // two per TMEM lane quarter, each half of the tile's columns
constexpr int ECOLS = TN / 2;       // columns per epilogue thread
constexpr int THREADS = 32 * EPI_WARPS + 64;   // + producer warp + MMA-issue warp
constexpr long SPIN = 1L << 22;     // polls before a wait gives up

static_assert(NDIAG * TN <= TMEM_COLS, "accumulators exceed TMEM");
static_assert(ECOLS % 4 == 0, "epilogue column groups of 4");
static_assert(NDIAG == 10 && DSUM == 11 && BITS == 6, "the epilogue pairs diagonals 2..11 into H (2..7) and L (8..11)");
// largest |sum of the digit products on one diagonal| per k: the two pairs
// with a leading digit (64 * 32 each) and the others (32 * 32), or 64 * 64
// (below 2^22 the epilogue converts them to integers with one fp32 add)
static_assert((long)KC * (2 * 64 * 32 + (DIG - 2) * 32 * 32) < (1L << 22), "diagonal sums must stay exact in fp32");
static_assert((long)KC * 64 * 64 < (1L << 22), "diagonal sums must stay exact in fp32");
static_assert(SMEM <= 227 * 1024, "shared memory ring too large");

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, leading byte
// offset (between core matrices adjacent in K) and stride byte offset
// (between core matrices adjacent in M / N), version bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase; gives up when another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort, long limit = SPIN) {
  for (long it = 0; it < limit; ++it) {
    if (mbar_try(bar, parity)) return true;
    if (*abort) return false;
    if (it > 32) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ inline double part_of(double v, int) { return v; }
__device__ inline double part_of(const cplx& v, int part) { return part ? v.im : v.re; }

// One real operand as rows x K: element (r, k) = part(X[rmap(r) * rs + kmap(k) * ks]).
template <typename T>
struct Src {
  BOp<T> X;
  IMap rmap, kmap;
  int64_t rs = 1, ks = 1;
};

// exponent e of a row (max |x| < 2^e) from its biased maximum exponent
__device__ __forceinline__ int row_exp(int evm) { return evm ? evm - 1022 : 0; }

// The operands of one product call (A and B) as rows x K, cut into digit
// blocks with row tiles of TR rows.  A complex operand yields the digits of
// its real part in out and of its imaginary part in out2, both scaled by one
// power of two per row (above the row's largest |re| or |im|), so that the
// products of both parts can share accumulators.
constexpr int MAXOPS = 4;
template <typename T>
struct SplitSet {
  Src<T> s[MAXOPS];
  int R[MAXOPS], TR[MAXOPS], RT[MAXOPS];
  uint8_t* out[MAXOPS];
  uint8_t* out2[MAXOPS];  // imaginary part's digits (complex operands)
  int* ex[MAXOPS];    // biased exponent of each row's largest |entry| (0: zero row)
  int items[MAXOPS];  // batch items to cut: 1 for an operand shared by every item
};

__device__ __forceinline__ unsigned long long mag_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFull;
}
__device__ __forceinline__ unsigned long long mag_bits(const cplx& v) {
  return max(mag_bits(v.re), mag_bits(v.im));
}

// Balanced base-64 digits of v 2^{FRAC - e} rounded to an integer, as bf16
// values, for the 8 consecutive k of one 16-byte row segment of a block:
// blk points at digit 0's segment; digit p lies BLK bytes further.
__device__ __forceinline__ void put_digits(const double (&v)[8], int e, uint8_t* blk, int BLK) {
  int dg[8][DIG];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v[c]);
    const int ev = (int)((u >> 52) & 0x7FF);
    // |v| 2^{FRAC - e} rounded to an integer (<= 2^FRAC), then signed
    const long long m = (long long)((u & 0xFFFFFFFFFFFFFull) | (1ull << 52));
    const int sh = ev - (1075 - FRAC) - e;
    long long x = 0;
    if (ev != 0) {
      if (sh >= 0) x = m << sh;
      else if (sh > -62) x = ((m >> (-sh - 1)) + 1) >> 1;
    }
    if (u >> 63) x = -x;
    // balanced base-64 digits, least significant first, in 32-bit halves:
    // x = hi 2^30 + lo with 0 <= lo < 2^30.  A digit is d = (t & 63) - 32
    // with t = v + 32, and the rest is (v - d) / 64 = t >> 6.  Five digits
    // of lo leave a carry of 0 or 1 into hi; four of hi leave the leading
    // digit (|.| <= 64).
    int lo = (int)(x & 0x3FFFFFFFll), hi = (int)(x >> 30);
#pragma unroll
    for (int p = DIG - 1; p >= DIG - 5; --p) {
      const int t = lo + 32;
      dg[c][p] = (t & 63) - 32;
      lo = t >> BITS;
    }
    hi += lo;
#pragma unroll
    for (int p = DIG - 6; p > 0; --p) {
      const int t = hi + 32;
      dg[c][p] = (t & 63) - 32;
      hi = t >> BITS;
    }
    dg[c][0] = hi;
  }
#pragma unroll
  for (int p = 0; p < DIG; ++p) {
    uint32_t w[4];
#pragma unroll
    for (int c = 0; c < 8; c += 2) {
      // d (|d| <= 64) as an exact float: 1.5 * 2^23 + d has d in its low
      // mantissa bits; subtracting 1.5 * 2^23 leaves d, whose upper 16
      // bits are its bf16 encoding (d has at most 7 significant bits)
      const float f0 = __int_as_float(0x4B400000 + dg[c][p]) - 12582912.0f;
      const float f1 = __int_as_float(0x4B400000 + dg[c + 1][p]) - 12582912.0f;
      w[c >> 1] = __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632);
    }
    *reinterpret_cast<uint4*>(blk + (int64_t)p * BLK) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// One launch for all operands: CTA = 32 rows x 8 warps; warp w takes the
// 8-deep k groups w, w+8, ...  Pass 1 finds each row's largest magnitude
// (compared as bit patterns, which order like the values; over both parts
// of a complex row), pass 2 writes the balanced base-64 digits of the row
// scaled by 2^{FRAC - e}, rounded to an integer (both parts of a complex
// row from one read).
template <typename T>
__global__ void __launch_bounds__(256) k_split(SplitSet<T> ss, int K, int KT, int b0, int nb) {
  const int op = blockIdx.z / nb, bl = blockIdx.z % nb, b = b0 + bl;
  const int R = ss.R[op], TR = ss.TR[op], Rpad = ss.RT[op] * TR;
  if (blockIdx.x * 32 >= Rpad || bl >= ss.items[op]) return;  // uniform over the CTA
  const Src<T>& s = ss.s[op];
  const int lr = threadIdx.x & 31, kw = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + lr;
  const T* X = s.X.item(b);
  const bool live = r < R;
  const int64_t roff = live ? (int64_t)s.rmap.at(b, r) * s.rs : 0;
  const int ngrp = KT * 2;
  __shared__ unsigned long long smax[8][32];
  unsigned long long mx = 0;
  if (live)
    for (int gi = kw; gi < ngrp; gi += 8)
      for (int c = 0; c < 8; ++c) {
        const int k = gi * 8 + c;
        if (k >= K) break;
        mx = max(mx, mag_bits(X[roff + (int64_t)s.kmap.at(b, k) * s.ks]));
      }
  smax[kw][lr] = mx;
  __syncthreads();
#pragma unroll
  for (int w = 0; w < 8; ++w) mx = max(mx, smax[w][lr]);
  const int evm = (int)(mx >> 52);
  if (kw == 0 && r < Rpad) ss.ex[op][(int64_t)bl * Rpad + r] = evm;
  if (r >= Rpad) return;
  const bool zero = evm == 0;
  const int e = row_exp(evm);
  const int BLK = TR * TK * 2;
  const int tile = r / TR, rr = r % TR;
  const int64_t rowoff = ((int64_t)bl * ss.RT[op] + tile) * KT * (int64_t)(DIG * BLK) + (rr >> 3) * 256 + (rr & 7) * 16;
  for (int gi = kw; gi < ngrp; gi += 8) {
    const int k0 = gi * 8;
    T xv[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int k = k0 + c;
      xv[c] = (live && !zero && k < K) ? X[roff + (int64_t)s.kmap.at(b, k) * s.ks] : T(0.0);
    }
    const int64_t boff = rowoff + (int64_t)(k0 >> 4) * (DIG * BLK) + ((k0 >> 3) & 1) * 128;
    double v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = part_of(xv[c], 0);
    put_digits(v, e, ss.out[op] + boff, BLK);
    if constexpr (std::is_same<T, cplx>::value) {
#pragma unroll
      for (int c = 0; c < 8; ++c) v[c] = part_of(xv[c], 1);
      put_digits(v, e, ss.out2[op] + boff, BLK);
    }
  }
}

__device__ __noinline__ double scale_slow(long long R, int es) { return ldexp((double)R, es); }

// R 2^es as the nearest double (ties to even), from the integer's bits;
// falls back to ldexp outside the normal range.
__device__ __forceinline__ double fixed_to_double(long long R, int es) {
  if (R == 0) return 0.0;
  const unsigned long long sgn = R < 0 ? (1ull << 63) : 0ull;
  unsigned long long a = R < 0 ? (unsigned long long)(-R) : (unsigned long long)R;
  const int lz = __clzll((long long)a);
  a <<= lz;                                    // leading one at bit 63
  unsigned long long m = a >> 11;              // 53 significant bits
  const unsigned long long rem = a & 0x7FFull;
  m += (rem > 0x400ull || (rem == 0x400ull && (m & 1ull))) ? 1ull : 0ull;
  const int e2 = es + 63 - lz;                 // value in [2^e2, 2^(e2+1))
  if (e2 + 1023 < 1 || e2 + 1023 > 2046) return scale_slow(R, es);
  // m carries the hidden bit: adding it to (exponent - 1) sets the exponent
  // (and carries once more when rounding reached 2^53)
  return __longlong_as_double((long long)(sgn | (((unsigned long long)(e2 + 1022) << 52) + m)));
}

template <typename T>
struct GemmP {
  const uint8_t* As;
  const uint8_t* Bs;
  // two products into the same accumulators (the two terms of one component
  // of a complex product): after the KT k steps of As Bs, KT more of
  // As2 Bs2, negated when neg2 (the operands of both share their row scales)
  const uint8_t* As2;
  const uint8_t* Bs2;
  int pair, neg2;
  const int* ea;
  const int* eb;
  int MT, NT, KT, M, N;
  int lsb;             // fraction bits of the fixed-point result
  double alpha, beta;
  int amode;                 // 1: alpha = +-1 (applied as a sign flip)
  long long asign;           // sign bit to flip when amode = 1
  BOp<T> C;
  IMap crow;
  int cpart;           // complex C: component written (0 re, 1 im)
  int b0;              // first batch item of this launch
  int a_bl, b_bl;      // 1, or 0 for an operand whose digits serve every item
  int nitems;          // batch items of this launch (tiles: MT NT nitems)
  unsigned* err;
};

template <typename T, bool BETA0, bool TRANS>
__global__ void __launch_bounds__(THREADS, 1) k_gemm_tc(GemmP<T> g) {
  // Persistent: CTA c takes the tiles c, c + gridDim.x, ... of the launch
  // (tile t = item t / (MT NT), then row tile, then column tile), so that the
  // next tile's copies and products overlap this tile's epilogue and the
  // TMEM allocation and barrier set-up happen once per CTA.  The stage ring,
  // the accumulator hand-over (acc_full / acc_empty) and their phases run on
  // across tiles.
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t full[NST], empty[NST], acc_full, acc_empty;
  __shared__ int s_eb[TN];
  __shared__ uint32_t tslot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_item = g.MT * g.NT;
  const int ntiles = tiles_item * g.nitems;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i < NST; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty[i])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&acc_full)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&acc_empty)), "r"(32 * EPI_WARPS));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tslot;
  volatile int* abrt = &abort_flag;
  const int KTV = g.pair ? 2 * g.KT : g.KT;   // k steps of a tile (both products of a pair)
  const int nchunk = (KTV + KCT - 1) / KCT;
  const uint32_t sbase = su32(smem);

  if (warp == EPI_WARPS) {
    // producer: one bulk copy per operand per k step, the ring running on
    // across tiles
    if (lane == 0) {
      long it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int bl = t / tiles_item, rem = t % tiles_item;
        const int mt = rem % g.MT, nt = rem / g.MT;
        const int64_t a_off = ((int64_t)(bl * g.a_bl) * g.MT + mt) * g.KT * (int64_t)ASTG;
        const int64_t b_off = ((int64_t)(bl * g.b_bl) * g.NT + nt) * g.KT * (int64_t)BSTG;
        for (int vk = 0; vk < KTV; ++vk, ++it) {
          const bool second = vk >= g.KT;
          const int k = second ? vk - g.KT : vk;
          const uint8_t* a_src = (second ? g.As2 : g.As) + a_off;
          const uint8_t* b_src = (second ? g.Bs2 : g.Bs) + b_off;
          const int s = (int)(it % NST);
          if (it >= NST && !mbar_wait(su32(&empty[s]), (int)((it / NST) & 1) ^ 1, abrt)) {
            ok = false;
            break;
          }
          const uint32_t fb = su32(&full[s]), dst = sbase + s * STAGE;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(STAGE) : "memory");
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                       ::"r"(dst), "l"(a_src + (int64_t)k * ASTG), "r"(ASTG), "r"(fb) : "memory");
          asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                       ::"r"(dst + ASTG), "l"(b_src + (int64_t)k * BSTG), "r"(BSTG), "r"(fb) : "memory");
        }
      }
      if (!ok) {
        *abrt = 1;
        atomicOr(g.err, DEV_ERR_TIMEOUT);
      }
    }
  } else if (warp == EPI_WARPS + 1) {
    // MMA issue: 55 digit-pair products per k step into the 10 diagonal accumulators
    if (lane == 0) {
      // B's digit blocks lie one after another with the same row-group stride,
      // so digits q0 .. q0+n-1 form one operand of n * 48 rows, and A_p times
      // it lands in the accumulators of diagonals p+q0 .. p+q0+n-1, which are
      // adjacent in TMEM: one MMA (N <= 240) per (p, group of <= 5 digits).
      const uint32_t idesc0 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TM >> 4) << 24);
      long it = 0, cc = 0;   // k steps and accumulator chunks issued so far
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int kk = 0;
        for (int c = 0; c < nchunk && ok; ++c, ++cc) {
          // the epilogue has read the previous chunk's accumulators
          if (cc > 0 && !mbar_wait(su32(&acc_empty), (int)((cc - 1) & 1), abrt)) { ok = false; break; }
          fence_after();
          const int kend = min(KTV, (c + 1) * KCT);
          const int kbeg = kk;
          for (; kk < kend; ++kk, ++it) {
            const int s = (int)(it % NST);
            if (!mbar_wait(su32(&full[s]), (int)((it / NST) & 1), abrt)) { ok = false; break; }
            fence_after();
            const uint32_t a0 = sbase + s * STAGE, b0 = a0 + ASTG;
            // the second product of a pair enters negated: negate-B bit of the
            // instruction descriptor
            const uint32_t ineg = (g.neg2 && kk >= g.KT) ? (1u << 14) : 0u;
#pragma unroll
            for (int p = 0; p < DIG; ++p) {
              const uint64_t ad = sdesc(a0 + p * ABLK, 128, 256);
              const int nq_all = (DSUM - 1 - p) < DIG ? (DSUM - 1 - p) : DIG;   // q = 0 .. nq_all-1
#pragma unroll
              for (int q0 = 0; q0 < nq_all; q0 += QGRP) {
                const int nq = (nq_all - q0) < QGRP ? (nq_all - q0) : QGRP;
                // the first k step of a chunk overwrites: p = 0 covers every diagonal once
                const uint32_t acc = (kk != kbeg || p != 0) ? 1u : 0u;
                const uint64_t bd = sdesc(b0 + q0 * BBLK, 128, 256);
                const uint32_t idesc = idesc0 | ineg | ((uint32_t)((nq * TN) >> 3) << 17);
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + (uint32_t)((p + q0) * TN)),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
              }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&empty[s]))
                         : "memory");
          }
          if (!ok) break;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                           su32(&acc_full))
                       : "memory");
        }
      }
      if (!ok) {
        *abrt = 1;
        atomicOr(g.err, DEV_ERR_TIMEOUT);
      }
    }
  } else {
    // epilogue: warp w reads TMEM lane quarter w % 4 (its rows) and column
    // half w / 4; thread = row, 24 fixed-point sums.  While the MMAs run, the
    // C tile (beta != 0) and the columns' exponents are staged in shared
    // memory with asynchronous copies.  A transposed tile (rows of C^T are
    // C's columns) is staged and stored by all epilogue threads with the tile
    // column fastest, so that its global accesses stay coalesced, and each
    // thread's results pass through shared memory.  Every epilogue thread
    // runs the same tiles and the same named barriers; after a wait gives up
    // it skips the remaining waits and stores but still takes the barriers.
    const int quarter = warp & 3, c0 = (warp >> 2) * ECOLS;
    const int row = quarter * 32 + lane;
    double* s_c = reinterpret_cast<double*>(smem + NST * STAGE);
    constexpr int SLD = TRANS ? TMP : TM;   // staging stride
    constexpr int W = (int)(sizeof(T) / sizeof(double));
    const int etid = threadIdx.x;   // 0 .. 32 * EPI_WARPS - 1
    // diagonal d = di + 2 has weight 2^{-6d}; R counts units of 2^{-lsb}.
    // Adjacent diagonals pair up exactly in 32 bits (y = x_d * 64 + x_{d+1},
    // |y| < 2^29), the pairs of d = 2..7 form H (units 2^{-42}) and those of
    // d = 8..11 form L (units 2^{-66}) in 64 bits; H enters R exactly and L
    // rounded once.  lsb is at least 42 (K <= 2^20).
    const int shH = g.lsb - 42, shL = 66 - g.lsb;
    const long long halfL = 1ll << (shL - 1);
    const bool amode1 = g.amode == 1, beta1 = g.beta == 1.0;
    bool ok = true;
    long cc = 0;   // accumulator chunks consumed so far
    bool first = true;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      const int bl = t / tiles_item, rem = t % tiles_item;
      const int mt = rem % g.MT, nt = rem / g.MT;
      const int i = mt * TM + row;
      const int b = g.b0 + bl;
      double* Cb = reinterpret_cast<double*>(g.C.item(b));
      const int64_t ci = (!TRANS && i < g.M) ? (int64_t)g.crow.at(b, i) : 0;
      // the previous tile's conversion has finished with s_eb and s_c
      if (!first) asm volatile("bar.sync 1, %0;" ::"r"(32 * EPI_WARPS) : "memory");
      first = false;
      if (threadIdx.x < TN)
        s_eb[threadIdx.x] = nt * TN + threadIdx.x < g.N ? row_exp(g.eb[(int64_t)(bl * g.b_bl) * g.NT * TN + nt * TN + threadIdx.x]) : 0;
      // the old C values of a normal tile go straight to registers (issued
      // now, they arrive while the products finish); a transposed tile's are
      // staged in shared memory, tile column fastest
      double cold[ECOLS];
      if constexpr (!TRANS) {
        if (!BETA0 && ok && i < g.M) {
#pragma unroll
          for (int jj = 0; jj < ECOLS; ++jj) {
            const int col = nt * TN + c0 + jj;
            cold[jj] = col < g.N ? Cb[(ci + (int64_t)col * g.C.ld) * W + g.cpart] : 0.0;
          }
        }
      }
      if (!BETA0 && ok) {
        if constexpr (TRANS) {
          for (int e2 = etid; e2 < TM * TN; e2 += 32 * EPI_WARPS) {
            const int j = e2 % TN, r = e2 / TN;
            const int crw = nt * TN + j, ccol = mt * TM + r;
            if (crw < g.N && ccol < g.M)
              asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(su32(s_c + j * TMP + r)),
                           "l"(Cb + ((int64_t)g.crow.at(b, crw) + (int64_t)ccol * g.C.ld) * W + g.cpart)
                           : "memory");
          }
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
      long long R[ECOLS];
#pragma unroll
      for (int j = 0; j < ECOLS; ++j) R[j] = 0;
      for (int c = 0; c < nchunk; ++c, ++cc) {
        if (!ok) continue;
        if (!mbar_wait(su32(&acc_full), (int)(cc & 1), abrt)) { ok = false; continue; }
        fence_after();
#pragma unroll
        for (int cg = 0; cg < ECOLS / 4; ++cg) {
          uint32_t v[NDIAG][4];
#pragma unroll
          for (int di = 0; di < NDIAG; ++di) {
            const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(di * TN + c0 + cg * 4);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                         : "=r"(v[di][0]), "=r"(v[di][1]), "=r"(v[di][2]), "=r"(v[di][3])
                         : "r"(ta));
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // an fp32 holding an integer below 2^22, plus 1.5 * 2^23, has the
            // integer in its low mantissa bits: x = bits - 0x4B400000
            int y[NDIAG / 2];
#pragma unroll
            for (int k = 0; k < NDIAG / 2; ++k) {
              const uint32_t a = __float_as_uint(__uint_as_float(v[2 * k][j]) + 12582912.0f);
              const uint32_t c2 = __float_as_uint(__uint_as_float(v[2 * k + 1][j]) + 12582912.0f);
              y[k] = (int)(a * 64u + c2 - 65u * 0x4B400000u);
            }
            const long long H = ((long long)y[0] << 24) + ((long long)y[1] << 12) + (long long)y[2];
            const long long L = ((long long)y[3] << 12) + (long long)y[4];
            R[cg * 4 + j] += (H << shH) + ((L + halfL) >> shL);
          }
        }
        fence_before();
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&acc_empty)) : "memory");
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      asm volatile("bar.sync 1, %0;" ::"r"(32 * EPI_WARPS) : "memory");   // s_eb and s_c from other epilogue threads
      if (ok && i < g.M) {
        const int er = row_exp(g.ea[(int64_t)(bl * g.a_bl) * g.MT * TM + i]);
#pragma unroll
        for (int jj = 0; jj < ECOLS; ++jj) {
          const int j = c0 + jj;
          const int col = nt * TN + j;
          if (col >= g.N) break;
          double val = fixed_to_double(R[jj], er + s_eb[j] - g.lsb);
          double* sp = s_c + j * SLD + row;
          double c_old = 0.0;
          if constexpr (!BETA0) c_old = TRANS ? *sp : cold[jj];
          double out;
          if (amode1) {                // alpha = +-1: a sign flip
            val = __longlong_as_double(__double_as_longlong(val) ^ g.asign);
            if (BETA0) out = val;
            else if (beta1) out = c_old + val;
            else out = fma(g.beta, c_old, val);
          } else {
            if (BETA0) out = g.alpha * val;
            else out = fma(g.alpha, val, g.beta * c_old);
          }
          if constexpr (!TRANS) Cb[(ci + (int64_t)col * g.C.ld) * W + g.cpart] = out;
          else *sp = out;
        }
      }
      if constexpr (TRANS) {
        asm volatile("bar.sync 1, %0;" ::"r"(32 * EPI_WARPS) : "memory");
        if (ok)
          for (int e2 = etid; e2 < TM * TN; e2 += 32 * EPI_WARPS) {
            const int j = e2 % TN, r = e2 / TN;
            const int crw = nt * TN + j, ccol = mt * TM + r;
            if (crw < g.N && ccol < g.M)
              Cb[((int64_t)g.crow.at(b, crw) + (int64_t)ccol * g.C.ld) * W + g.cpart] = s_c[j * TMP + r];
          }
      }
    }
    if (!ok) {
      *abrt = 1;
      atomicOr(g.err, DEV_ERR_TIMEOUT);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

// digit pairs (p, q), 1 <= p, q <= DIG, with p + q <= DSUM
constexpr int npairs() {
  int n = 0;
  for (int p = 1; p <= DIG; ++p)
    for (int q = 1; q <= DIG; ++q) n += (p + q <= DSUM) ? 1 : 0;
  return n;
}
static_assert(npairs() == 55, "digit pair count");
static_assert(DIG == 10 && BITS == 6 && FRAC == 60, "the slicing splits 60 bits into 30 + 30");
static_assert(QGRP * TN <= 256 && (QGRP * TN) % 16 == 0, "MMA N for M = 128");

int ceil_log2(int64_t x) {
  int c = 0;
  while ((int64_t(1) << c) < x) ++c;
  return c;
}

template <typename T, bool BETA0, bool TRANS>
void set_smem_attr() {
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_gemm_tc<T, BETA0, TRANS>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
  });
}

struct Sizes {
  int MT, NT, KT;
  size_t a_item, b_item, ea_item, eb_item;
};

Sizes sizes(int M, int N, int K) {
  Sizes z;
  z.MT = (M + TM - 1) / TM;
  z.NT = (N + TN - 1) / TN;
  z.KT = (K + TK - 1) / TK;
  z.a_item = (size_t)z.MT * z.KT * ASTG;
  z.b_item = (size_t)z.NT * z.KT * BSTG;
  z.ea_item = (size_t)z.MT * TM * sizeof(int);
  z.eb_item = (size_t)z.NT * TN * sizeof(int);
  return z;
}

constexpr size_t WS_CAP = size_t(1) << 30;  // workspace bytes a launch group may use

}  // namespace tc

TcWorkspace*& tc_workspace() {
  static thread_local TcWorkspace* w = nullptr;
  return w;
}

size_t tc_workspace_cap() { return tc::WS_CAP; }

void tc_release(TcWorkspace* w) {
  if (w && w->p) dev_free(w->p, w->st);
  if (w) { w->p = nullptr; w->bytes = 0; }
}

// Fraction of the 128 x 48 output tiles that holds the product, in the
// better of the two orientations.
static double tile_fill(int M, int N) {
  using namespace tc;
  const double mn = (double)M * N;
  const double normal = (double)((M + TM - 1) / TM) * TM * ((N + TN - 1) / TN) * TN;
  const double trans = (double)((N + TM - 1) / TM) * TM * ((M + TN - 1) / TN) * TN;
  return mn / std::min(normal, trans);
}

// At most 8 rows against many columns and a long inner dimension.
static bool few_rows_long_k(int M, int N, int K) { return M <= 8 && N >= 32 && K >= 32; }

template <typename T>
bool tc_applicable(const GemmArgs<T>& g) {
  const TcWorkspace* w = tc_workspace();
  if (!w || !w->enabled || !w->err_slot || !*w->err_slot || g.ta || g.K > (1 << 20)) return false;
  if (w->force) return true;
  // one side of at least 32 and the other of at least 16: the short side
  // goes to the 48-wide tile dimension (transposed tiling when M is short)
  if (std::min(g.M, g.N) < 1 || std::max(g.M, g.N) < 32 || g.K < 16) return false;
  if (std::min(g.M, g.N) < 16 && !few_rows_long_k(g.M, g.N, g.K)) return false;
  // a side below 32 fills at best two thirds of the 48-wide tile side: such
  // products go to the tensor cores only while the tiles stay over ~28 % full
  // (measured: 28 x 113 gains there, 28 x 57 loses) -- except products of
  // at most 8 rows, N >= 32 and K >= 32, which the FP64-pipe kernels run at
  // under half their rate (4 x 114 x 64: 0.14 TFLOP/s); few columns stay on
  // the FP64 pipe's skinny kernels
  if (std::min(g.M, g.N) < 32 && tile_fill(g.M, g.N) < 0.28 && !few_rows_long_k(g.M, g.N, g.K)) return false;
  // short inner dimensions: ten accumulators per output are read back for
  // little work, so small items stay on the FP64 pipe
  if (g.K < lu_tune(TUNE_TC_MIN_K) && (g.M < 512 || g.N < 512)) return false;
  if ((double)g.M * g.N * g.K * g.batch < 1.0e5 * lu_tune(TUNE_TC_MIN_WORK_REAL)) return false;
  return true;
}

template <>
bool tc_applicable<cplx>(const GemmArgs<cplx>& g) {
  const TcWorkspace* w = tc_workspace();
  if (!w || !w->enabled || !w->err_slot || !*w->err_slot || g.ta || g.K > (1 << 20)) return false;
  if (g.alpha.im != 0.0 || g.beta.im != 0.0) return false;
  if (w->force) return true;
  if (std::min(g.M, g.N) < 1 || std::max(g.M, g.N) < 32 || g.K < 16) return false;
  if (std::min(g.M, g.N) < 16 && !few_rows_long_k(g.M, g.N, g.K)) return false;
  if (std::min(g.M, g.N) < 32 && tile_fill(g.M, g.N) < 0.28 && !few_rows_long_k(g.M, g.N, g.K)) return false;
  if (g.K < lu_tune(TUNE_TC_MIN_K) && (g.M < 512 || g.N < 512)) return false;
  if ((double)g.M * g.N * g.K * g.batch < 1.0e5 * lu_tune(TUNE_TC_MIN_WORK_CPLX)) return false;
  return true;
}

namespace {

cudaError_t ensure_ws(TcWorkspace* w, size_t bytes, cudaStream_t st) {
  if (w->bytes >= bytes) {
    if (w->st != st && w->p) {
      // the buffer moves to another stream: order it after its last use
      cudaError_t e = cudaStreamSynchronize(w->st);
      if (e != cudaSuccess) return e;
      w->st = st;
    }
    return cudaSuccess;
  }
  if (w->p) {
    cudaError_t e = cudaStreamSynchronize(w->st);
    if (e != cudaSuccess) return e;
    dev_free(w->p, st);
    w->p = nullptr;
    w->bytes = 0;
  }
  const size_t nb = std::max(bytes, (size_t)64 << 20);
  cudaError_t e = dev_malloc(&w->p, nb, st);
  if (e != cudaSuccess) { w->p = nullptr; return e; }
  w->bytes = nb;
  w->st = st;
  return cudaSuccess;
}

template <typename T>
void launch_split(const tc::SplitSet<T>& ss, int nops, int K, int KT, int b0, int nb, cudaStream_t st, Prof* pf) {
  int rmax = 0;
  for (int o = 0; o < nops; ++o) rmax = std::max(rmax, ss.RT[o] * ss.TR[o]);
  if (pf) {
    pf->begin(st);
    pf->note(rmax, nops, K, nb);
  }
  tc::k_split<T><<<dim3((rmax + 31) / 32, 1, nops * nb), 256, 0, st>>>(ss, K, KT, b0, nb);
  if (pf) pf->end(K_SPLIT, 0.0, st);
}

template <typename T>
void launch_mma(const tc::GemmP<T>& p, bool trans, int nb, int M, int N, int K, cudaStream_t st, Prof* pf) {
  if (pf) {
    pf->begin(st);
    pf->note(M, N, K, nb);
  }
  // persistent (from the tuned inner dimension on): at most one CTA per SM,
  // which the shared-memory ring and the TMEM accumulators allow anyway; else
  // one CTA per tile
  const int64_t ntiles = (int64_t)p.MT * p.NT * nb;
  const bool persist = K >= lu_tune(TUNE_TC_PERSIST_MIN_K);
  dim3 grid((unsigned)(persist ? std::min<int64_t>(ntiles, device_sms()) : ntiles));
  auto go = [&](auto beta0, auto trans) {
    constexpr bool B0 = decltype(beta0)::value, TR = decltype(trans)::value;
    tc::set_smem_attr<T, B0, TR>();
    tc::k_gemm_tc<T, B0, TR><<<grid, tc::THREADS, tc::SMEM, st>>>(p);
  };
  using t_ = std::true_type;
  using f_ = std::false_type;
  if (p.beta == 0.0) { if (trans) go(t_(), t_()); else go(t_(), f_()); }
  else { if (trans) go(f_(), t_()); else go(f_(), f_()); }
  // executed: bf16 tensor-core flops of the digit products over the padded
  // tiles; algorithmic: 2 M N K per real product (a pair holds two)
  const double npairs = tc::npairs();
  const double nprod = p.pair ? 2.0 : 1.0;
  const double exec = 2.0 * npairs * nprod * (double)p.MT * tc::TM * (double)p.NT * tc::TN * (double)p.KT * tc::TK * nb;
  if (pf) pf->end(K_GEMM_TC, 2.0 * nprod * M * (double)N * K * nb, st, exec);
}

}  // namespace

// An operand is the same matrix for every batch item when its items share
// one base and its index maps do not depend on the item (the leaf stage's
// Q and QH, for instance): its digits are then cut once and serve all items.
template <typename T>
bool shared_operand(const BOp<T>& X, const IMap& r, const IMap& k) {
  return !X.ptrs && X.stride == 0 && (X.div == 1 || X.sub == 0) && (!r.idx || r.period == 1) &&
         (!k.idx || k.period == 1);
}

// Orientation of the output tiles: C = A B in 128 x 48 tiles of C, or
// C^T = B^T A^T in 128 x 48 tiles of C^T (48-row tiles of C), the latter
// when it takes a quarter fewer waves of tiles over the SMs -- a product with few rows (the
// 32-row updates of the recursive LU and triangular solves, M = 32..64)
// wastes most of a 128-row tile but fits a 48-column one; a grid that fits
// in one wave either way stays in the normal form.
static bool tc_transposed(int M, int N, int batch) {
  using namespace tc;
  const int64_t sms = device_sms();
  const int64_t normal = (int64_t)((M + TM - 1) / TM) * ((N + TN - 1) / TN) * batch;
  const int64_t trans = (int64_t)((N + TM - 1) / TM) * ((M + TN - 1) / TN) * batch;
  // one CTA per SM: the time goes with the number of waves of tiles; the
  // transposed epilogue (staged through shared memory) costs more per tile,
  // so it has to save at least a quarter of the waves
  return 4 * ((trans + sms - 1) / sms) <= 3 * ((normal + sms - 1) / sms);
}

template <typename T>
cudaError_t gemm_tc(const GemmArgs<T>& g, cudaStream_t st, Prof* pf) {
  using namespace tc;
  constexpr int NP = std::is_same<T, cplx>::value ? 2 : 1;
  TcWorkspace* w = tc_workspace();
  const bool tr = tc_transposed(g.M, g.N, g.batch);
  // rows of the A slot (the 128-row tiles) and of the B slot (48-row tiles)
  const int Ma = tr ? g.N : g.M, Nb = tr ? g.M : g.N;
  const Sizes z = sizes(Ma, Nb, g.K);
  const bool shA = g.batch > 1 && shared_operand(g.A, g.arow, g.acol);
  const bool shB = g.batch > 1 && shared_operand(g.B, g.brow, IMap());
  const bool shSa = tr ? shB : shA, shSb = tr ? shA : shB;   // per slot
  // per item and slot: NP digit arrays and one exponent array (the parts of
  // a complex row share their scale)
  const size_t a_sz = NP * z.a_item + z.ea_item, b_sz = NP * z.b_item + z.eb_item;
  const size_t fixed = (shSa ? a_sz : 0) + (shSb ? b_sz : 0);
  const size_t per_item = std::max<size_t>((shSa ? 0 : a_sz) + (shSb ? 0 : b_sz), 1);
  // batch items per launch group: their digit slices stay within the cap
  // (small enough and they are still in L2 when the products read them)
  const size_t cap = std::min<size_t>(WS_CAP, (size_t)std::max(lu_tune(TUNE_TC_CHUNK_MB), 1) << 20);
  const size_t room = cap > fixed ? cap - fixed : 0;
  const int nb_max = (int)std::max<size_t>(1, std::min<size_t>(std::min(g.batch, 65535 / 2), room / per_item));
  const size_t na = shSa ? 1 : (size_t)nb_max, nbb = shSb ? 1 : (size_t)nb_max;
  cudaError_t e = ensure_ws(w, a_sz * na + b_sz * nbb, st);
  if (e != cudaSuccess) return e;
  uint8_t* base = static_cast<uint8_t*>(w->p);
  uint8_t* As[2] = {nullptr, nullptr};   // digits of the A slot, per real part
  uint8_t* Bs[2] = {nullptr, nullptr};
  int* ea;
  int* eb;
  {
    uint8_t* q = base;
    for (int pt = 0; pt < NP; ++pt) {
      As[pt] = q; q += z.a_item * na;
      Bs[pt] = q; q += z.b_item * nbb;
    }
    ea = reinterpret_cast<int*>(q); q += z.ea_item * na;
    eb = reinterpret_cast<int*>(q); q += z.eb_item * nbb;
  }
  // fixed-point fraction bits: a complex component sums 2K products
  const int lsb = 62 - ceil_log2(std::max(NP * g.K, 1));
  double alpha, beta;
  if constexpr (NP == 2) { alpha = g.alpha.re; beta = g.beta.re; }
  else { alpha = g.alpha; beta = g.beta; }
  for (int b0 = 0; b0 < g.batch; b0 += nb_max) {
    const int nb = std::min(nb_max, g.batch - b0);
    SplitSet<T> ss;
    // A (M x K) and B^T (N x K) as row sources
    Src<T> sa;
    sa.X = g.A; sa.rmap = g.arow; sa.kmap = g.acol; sa.rs = 1; sa.ks = g.A.ld;
    Src<T> sb;
    sb.X = g.B; sb.kmap = g.brow; sb.rs = g.B.ld; sb.ks = 1;
    ss.s[0] = tr ? sb : sa; ss.R[0] = Ma; ss.TR[0] = TM; ss.RT[0] = z.MT;
    ss.out[0] = As[0]; ss.out2[0] = As[1]; ss.ex[0] = ea;
    ss.items[0] = (shSa && b0 > 0) ? 0 : (shSa ? 1 : nb);  // a shared operand is cut once per call
    ss.s[1] = tr ? sa : sb; ss.R[1] = Nb; ss.TR[1] = TN; ss.RT[1] = z.NT;
    ss.out[1] = Bs[0]; ss.out2[1] = Bs[1]; ss.ex[1] = eb;
    ss.items[1] = (shSb && b0 > 0) ? 0 : (shSb ? 1 : nb);
    launch_split<T>(ss, 2, g.K, z.KT, b0, nb, st, pf);
    GemmP<T> p;
    p.MT = z.MT; p.NT = z.NT; p.KT = z.KT; p.M = Ma; p.N = Nb; p.lsb = lsb;
    p.C = g.C; p.crow = g.crow; p.b0 = b0; p.err = *w->err_slot;
    p.a_bl = shSa ? 0 : 1;
    p.b_bl = shSb ? 0 : 1;
    p.nitems = nb;
    p.ea = ea; p.eb = eb;
    p.alpha = alpha;
    p.beta = beta;
    p.amode = (alpha == 1.0 || alpha == -1.0) ? 1 : 0;
    p.asign = alpha == -1.0 ? (long long)(1ull << 63) : 0ll;
    if constexpr (NP == 1) {
      p.As = As[0]; p.Bs = Bs[0];
      p.As2 = nullptr; p.Bs2 = nullptr; p.pair = 0; p.neg2 = 0;
      p.cpart = 0;
      launch_mma<T>(p, tr, nb, g.M, g.N, g.K, st, pf);
    } else {
      // complex (real alpha, beta), each component one launch of two
      // products into the same accumulators:
      //   C.re = alpha (Ar Br - Ai Bi) + beta C.re,  C.im = alpha (Ar Bi + Ai Br) + beta C.im
      // (transposed, the A slot holds B's parts and the B slot A's)
      uint8_t* const* Ap = tr ? Bs : As;   // digits of A's parts
      uint8_t* const* Bp = tr ? As : Bs;   // digits of B's parts
      auto slots = [&](int a_part, int b_part, const uint8_t*& sa_d, const uint8_t*& sb_d) {
        sa_d = tr ? Bp[b_part] : Ap[a_part];
        sb_d = tr ? Ap[a_part] : Bp[b_part];
      };
      p.pair = 1;
      slots(0, 0, p.As, p.Bs);
      slots(1, 1, p.As2, p.Bs2);
      p.neg2 = 1;
      p.cpart = 0;
      launch_mma<T>(p, tr, nb, g.M, g.N, g.K, st, pf);
      slots(0, 1, p.As, p.Bs);
      slots(1, 0, p.As2, p.Bs2);
      p.neg2 = 0;
      p.cpart = 1;
      launch_mma<T>(p, tr, nb, g.M, g.N, g.K, st, pf);
    }
  }
  return cudaGetLastError();
}

// Bounded-wait check (hps_debug_wait_timeout, which 2): one CTA waits with
// the pipeline's mbarrier wait on phase 0 of a barrier that expects one
// arrival; nothing arrives unless `satisfied`.  A wait that gives up sets
// DEV_ERR_TIMEOUT in *err.
__global__ void k_debug_mbar_wait(int satisfied, long limit, unsigned* err) {
  using namespace tc;
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (satisfied) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(&bar)) : "memory");
    if (!mbar_wait(su32(&bar), 0, &abort_flag, limit)) atomicOr(err, DEV_ERR_TIMEOUT);
  }
}

cudaError_t debug_mbar_wait(int satisfied, long limit, unsigned* err, cudaStream_t st) {
  k_debug_mbar_wait<<<1, 32, 0, st>>>(satisfied, limit, err);
  return cudaGetLastError();
}

template bool tc_applicable<double>(const GemmArgs<double>&);
template cudaError_t gemm_tc<double>(const GemmArgs<double>&, cudaStream_t, Prof*);
template cudaError_t gemm_tc<cplx>(const GemmArgs<cplx>&, cudaStream_t, Prof*);

}  // namespace hps
