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

// returns false if the barrier timed out (status already set)
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned int g = ld_volatile_u32(&bar->gen);
    __threadfence();
    unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long spins = 0;
      while (ld_volatile_u32(&bar->gen) == g) {
        __nanosleep(64);
        if (++spins > (1ll << 25)) {  // ~2 s at >= 64 ns per spin
          set_status(status, CBC_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        if ((spins & 1023) == 0 && *((volatile int*)status) == CBC_ERR_TIMEOUT) {
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// warp / block reductions -----------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ zdbl warp_sum(zdbl v) {
  return {warp_sum(v.re), warp_sum(v.im)};
}

}  // namespace cbc
