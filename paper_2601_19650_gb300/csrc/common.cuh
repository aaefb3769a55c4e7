// Shared device helpers of the CBC library: scalar types, complex arithmetic, the
// device status word and a bounded grid barrier for cooperative launches.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cbc.h"

namespace cbc {

// ----------------------------------------------------------------------------------
// scalars: real double and complex double share one set of helpers so every FP64
// kernel is written once as a template.
// ----------------------------------------------------------------------------------
struct zdbl {
  double re, im;
};

__host__ __device__ __forceinline__ zdbl mkz(double r, double i) { return zdbl{r, i}; }
__host__ __device__ __forceinline__ zdbl operator+(zdbl a, zdbl b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ zdbl operator-(zdbl a, zdbl b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ zdbl operator*(zdbl a, zdbl b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__host__ __device__ __forceinline__ zdbl operator*(double s, zdbl a) { return {s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ zdbl operator-(zdbl a) { return {-a.re, -a.im}; }

template <typename T> struct ops;

template <> struct ops<double> {
  static constexpr bool cplx = false;
  __host__ __device__ static __forceinline__ double zero() { return 0.0; }
  __host__ __device__ static __forceinline__ double one() { return 1.0; }
  __host__ __device__ static __forceinline__ double conj(double a) { return a; }
  __host__ __device__ static __forceinline__ double real(double a) { return a; }
  __host__ __device__ static __forceinline__ double imag(double) { return 0.0; }
  __host__ __device__ static __forceinline__ double abs2(double a) { return a * a; }
  __host__ __device__ static __forceinline__ double make(double r, double) { return r; }
  __host__ __device__ static __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
  __host__ __device__ static __forceinline__ double scale(double s, double a) { return s * a; }
};

template <> struct ops<zdbl> {
  static constexpr bool cplx = true;
  __host__ __device__ static __forceinline__ zdbl zero() { return {0.0, 0.0}; }
  __host__ __device__ static __forceinline__ zdbl one() { return {1.0, 0.0}; }
  __host__ __device__ static __forceinline__ zdbl conj(zdbl a) { return {a.re, -a.im}; }
  __host__ __device__ static __forceinline__ double real(zdbl a) { return a.re; }
  __host__ __device__ static __forceinline__ double imag(zdbl a) { return a.im; }
  __host__ __device__ static __forceinline__ double abs2(zdbl a) { return a.re * a.re + a.im * a.im; }
  __host__ __device__ static __forceinline__ zdbl make(double r, double i) { return {r, i}; }
  // a*b + c
  __host__ __device__ static __forceinline__ zdbl fma(zdbl a, zdbl b, zdbl c) {
    return {::fma(a.re, b.re, ::fma(-a.im, b.im, c.re)), ::fma(a.re, b.im, ::fma(a.im, b.re, c.im))};
  }
  __host__ __device__ static __forceinline__ zdbl scale(double s, zdbl a) { return {s * a.re, s * a.im}; }
};

// ----------------------------------------------------------------------------------
// device status word: kernels never trap; they record the first error and return.
// ----------------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ----------------------------------------------------------------------------------
// grid barrier for cooperative launches (all CTAs co-resident by construction).
// Every wait is bounded: after ~2 s without progress the barrier records
// CBC_ERR_TIMEOUT and lets the caller return.
// ----------------------------------------------------------------------------------
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int* p) {
  return *((volatile const unsigned int*)p);
}

// Spin until the 32-bit word at p differs from `seen`, for at most `limit` SM clock
// cycles (clock64).  Returns true when it changed; on time-out records CBC_ERR_TIMEOUT
// in *status and returns false.  Also gives up (false) as soon as another thread has
// recorded a time-out.  Every device-side wait of the library has this shape: no wait
// runs unbounded, and a kernel that gave up returns so the host can read the status.
__device__ __forceinline__ bool wait_word_change(const unsigned int* p, unsigned int seen,
                                                 int* status, long long limit) {
  const long long t0 = clock64();
  unsigned int cur;
  while (true) {
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(p) : "memory");
    if (cur != seen) return true;
    if (clock64() - t0 > limit) {
      set_status(status, CBC_ERR_TIMEOUT);
      return false;
    }
    if (status && *((volatile int*)status) == CBC_ERR_TIMEOUT) return false;
  }
}

constexpr long long kBarrierWaitCycles = 4000000000LL;  // ~2 s at the boost clock

// returns false if the barrier timed out (status already set).  Arrival is a release
// add at GPU scope, waiting an acquire load of the generation word.
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, int* status,
                                          unsigned int nctas = 0) {
  if (nctas == 0) nctas = gridDim.x;  // else: the CTAs of one group (cluster) of a batch
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned int g, arrived;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(&bar->gen) : "memory");
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;"
                 : "=r"(arrived)
                 : "l"(&bar->count)
                 : "memory");
    if (arrived == nctas - 1) {
      asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(&bar->count) : "memory");
      asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&bar->gen) : "memory");
    } else {
      ok = wait_word_change(&bar->gen, g, status, kBarrierWaitCycles) ? 1 : 0;
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// 1/x for finite nonzero x by Newton-Raphson on f(r) = 1/r - x, r <- r (2 - x r),
// started from the single-precision reciprocal of the mantissa (the exponent is split
// off with frexp so any double works): ~23 -> 46 -> 92 correct bits.  Used where a
// long dependent chain of FP64 divisions would otherwise dominate the latency.
__device__ __forceinline__ double rcp64(double x) {
  int ex;
  double f = frexp(x, &ex);
  double r = (double)__frcp_rn((float)f);
  r = fma(r, fma(-f, r, 1.0), r);
  r = fma(r, fma(-f, r, 1.0), r);
  return ldexp(r, -ex);
}

// 1/sqrt(x) for finite x > 0 by Newton-Raphson on f(r) = 1/r^2 - x,
// r <- r (3 - x r^2) / 2, seeded with the single-precision reciprocal square root of
// the mantissa (an even exponent is split off): ~23 -> 46 -> 92 correct bits in six
// dependent FP64 operations.
__device__ __forceinline__ double rsqrt64(double x) {
  int ex;
  double f = frexp(x, &ex);  // x = f 2^ex, f in [0.5, 1)
  if (ex & 1) {              // make the exponent even
    f *= 2.0;
    ex -= 1;
  }
  double r = (double)rsqrtf((float)f);
  double h = 0.5 * f;
  r = r * fma(-h * r, r, 1.5);
  r = r * fma(-h * r, r, 1.5);
  return ldexp(r, -ex / 2);
}

// Row i of entry t of a packed lower triangle (t = i (i + 1) / 2 + c, 0 <= c <= i).  The
// estimate comes from a single-precision square root (FP64 throughput per SM is two
// orders of magnitude below FP32 on this part) and is corrected in integer arithmetic.
__device__ __forceinline__ int tri_row(int64_t t) {
  int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((int64_t)(i + 1) * (i + 2) / 2 <= t) ++i;
  while ((int64_t)i * (i + 1) / 2 > t) --i;
  return i;
}

// warp / block reductions -----------------------------------------------------------
__device__ __forceinline__ double shfl_xor(double v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ zdbl shfl_xor(zdbl v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.re, o), __shfl_xor_sync(0xffffffffu, v.im, o)};
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ zdbl warp_sum(zdbl v) {
  return {warp_sum(v.re), warp_sum(v.im)};
}

}  // namespace cbc
