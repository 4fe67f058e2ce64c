// Shared device-side helpers: a complex<double> value type, scalar traits and
// a bounded inter-CTA barrier for cooperative launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hps {

struct cplx {
  double re, im;
  __host__ __device__ cplx() : re(0.0), im(0.0) {}
  __host__ __device__ cplx(double r) : re(r), im(0.0) {}
  __host__ __device__ cplx(double r, double i) : re(r), im(i) {}
};

__host__ __device__ inline cplx operator+(cplx a, cplx b) { return cplx(a.re + b.re, a.im + b.im); }
__host__ __device__ inline cplx operator-(cplx a, cplx b) { return cplx(a.re - b.re, a.im - b.im); }
__host__ __device__ inline cplx operator-(cplx a) { return cplx(-a.re, -a.im); }
__host__ __device__ inline bool operator==(cplx a, cplx b) { return a.re == b.re && a.im == b.im; }
__host__ __device__ inline cplx operator*(cplx a, cplx b) {
  return cplx(fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re));
}

// Scalar traits: fused multiply-add acc + a*b, magnitude used for pivoting
// (|re| + |im| for complex, no square root), reciprocal and zero test.
__host__ __device__ inline double fmac(double acc, double a, double b) { return fma(a, b, acc); }
__host__ __device__ inline cplx fmac(cplx acc, cplx a, cplx b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc - a*b
__host__ __device__ inline double fmsc(double acc, double a, double b) { return fma(-a, b, acc); }
__host__ __device__ inline cplx fmsc(cplx acc, cplx a, cplx b) {
  acc.re = fma(-a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
__host__ __device__ inline double mag1(double a) { return fabs(a); }
__host__ __device__ inline double mag1(cplx a) { return fabs(a.re) + fabs(a.im); }
__host__ __device__ inline double recip(double a) { return 1.0 / a; }
__host__ __device__ inline cplx recip(cplx a) {
  // 1/(x+iy) = (x - iy)/(x^2+y^2).  On the device x and y are first scaled by
  // the power of two 2^-e that brings max(|x|, |y|) into [1, 2) (exact), so
  // that the squared magnitude can neither overflow nor underflow and one
  // division suffices (the FP64 pipe is the scarce unit here); extreme
  // exponents, and the host, scale by the larger component instead.
#ifdef __CUDA_ARCH__
  const double s = fmax(fabs(a.re), fabs(a.im));
  const int eb = (int)((__double_as_longlong(s) >> 52) & 0x7ff);   // biased exponent of s
  if (eb >= 64 && eb <= 1982) {
    const double sc = __longlong_as_double((long long)(2046 - eb) << 52);   // 2^(1023 - eb)
    const double xr = a.re * sc, xi = a.im * sc;
    const double r = sc / fma(xr, xr, xi * xi);
    return cplx(xr * r, -xi * r);
  }
#endif
  double s2 = fmax(fabs(a.re), fabs(a.im));
  double xr2 = a.re / s2, xi2 = a.im / s2;
  double d = s2 * (xr2 * xr2 + xi2 * xi2);
  return cplx(xr2 / d, -xi2 / d);
}
__host__ __device__ inline bool is_zero(double a) { return a == 0.0; }
__host__ __device__ inline bool is_zero(cplx a) { return a.re == 0.0 && a.im == 0.0; }
__host__ __device__ inline double conj_of(double a) { return a; }
__host__ __device__ inline cplx conj_of(cplx a) { return cplx(a.re, -a.im); }
__host__ __device__ inline double scale(double a, double s) { return a * s; }
__host__ __device__ inline cplx scale(cplx a, double s) { return cplx(a.re * s, a.im * s); }

// Load through L2 only (no L1): for values another CTA of the same launch
// has written and published with a fence and a flag.
__device__ inline double ld_cg(const double* p) { return __ldcg(p); }
__device__ inline cplx ld_cg(const cplx* p) {
  const double* q = reinterpret_cast<const double*>(p);
  return cplx(__ldcg(q), __ldcg(q + 1));
}

template <typename T> struct zero_of { __host__ __device__ static T get() { return T(0.0); } };

// Error flag bits written by kernels into a device status word.
enum : unsigned {
  DEV_ERR_SINGULAR = 1u,
  DEV_ERR_TIMEOUT = 2u,
};

// Bounded barrier for the G co-resident CTAs of one group (cooperative
// launch).  bar[0] = arrival count, bar[1] = generation.  Gives up after
// `limit` polls, sets DEV_ERR_TIMEOUT in *err and returns false; callers then
// leave the kernel.  Every CTA of the group must call it the same number of
// times.
__device__ inline bool group_barrier(unsigned* bar, unsigned G, unsigned* err,
                                     unsigned long long limit = 20000000ull) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = bar + 1;
    unsigned gen = *vgen;
    __threadfence();
    unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == G - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long it = 0;
      while (*vgen == gen) {
        if (++it > limit) {
          atomicOr(err, DEV_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        if (*((volatile unsigned*)err) & DEV_ERR_TIMEOUT) { ok = 0; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Bounded wait until *f == want (another CTA publishes it with a fence).
// Gives up after `limit` polls and returns false; the caller records the
// timeout in its status word and leaves.
__device__ inline bool wait_flag(const volatile unsigned* f, unsigned want, unsigned long long limit) {
  unsigned long long it = 0;
  while (*f != want) {
    if (++it > limit) return false;
    __nanosleep(32);
  }
  return true;
}

}  // namespace hps
