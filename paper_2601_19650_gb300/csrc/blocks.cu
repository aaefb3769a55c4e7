// Building blocks of the sweeps exposed through the C ABI (cbc_heev, cbc_cholqr2) and
// device self-tests of primitives the kernels rely on (cbc_selftest_math,
// cbc_selftest_wait).  They run the same kernels as cbc_apply; tests use them to check
// each stage on its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels.cuh"
#include "planner.h"

namespace cbc {
namespace {

// out[4 i .. 4 i + 3] = rcp64(x_i), 1.0 / x_i, rsqrt64(x_i), rsqrt(x_i)
__global__ void math_selftest_kernel(const double* x, double* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    out[4 * i + 0] = rcp64(v);
    out[4 * i + 1] = 1.0 / v;
    out[4 * i + 2] = (v > 0.0) ? rsqrt64(v) : 0.0;
    out[4 * i + 3] = (v > 0.0) ? rsqrt(v) : 0.0;
  }
}

// one thread waits for a word that nothing writes; the wait gives up after `limit`
// clock cycles and records CBC_ERR_TIMEOUT in *status
__global__ void wait_selftest_kernel(const unsigned int* word, int* status, long long limit,
                                     int* returned) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const bool changed = wait_word_change(word, 0u, status, limit);
    *returned = changed ? 2 : 1;
  }
}

template <typename T>
int heev_t(int m, int kmax, int nb, T* A, double* lam, T* U, bool mixed, cudaStream_t s) {
  int* ints = nullptr;
  void* work = nullptr;
  const size_t wb = eig_workspace_bytes(m, kmax, ops<T>::cplx);
  cudaError_t e = pool_malloc(reinterpret_cast<void**>(&ints), sizeof(int) * (1 + nb), s);
  if (e != cudaSuccess) return cuda_fail(e, "cbc_heev: alloc");
  e = pool_malloc(&work, wb * nb, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(ints, s);
    return cuda_fail(e, "cbc_heev: alloc");
  }
  e = cudaMemsetAsync(ints, 0, sizeof(int) * (1 + nb), s);
  if (e == cudaSuccess)
    e = heev_top<T>(A, m, kmax, kmax, 0.0, -1.0, lam, U, ints + 1, work, ints, num_sms(), s, nb,
                    false, mixed);
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, ints, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(work, s);
  cudaFreeAsync(ints, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cbc_heev");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cbc_heev: synchronize");
  if (hs != 0) return fail(hs, "cbc_heev: device status %d", hs);
  return CBC_OK;
}

template <typename T>
int cholqr2_t(int m, int n, int nb, T* S, cudaStream_t s) {
  T* G = nullptr;
  int* status = nullptr;
  void* bar = nullptr;
  double* rn = nullptr;
  cudaError_t e = pool_malloc(reinterpret_cast<void**>(&G), sizeof(T) * (size_t)m * m * nb, s);
  if (e == cudaSuccess) e = pool_malloc(reinterpret_cast<void**>(&status), sizeof(int), s);
  if (e == cudaSuccess) e = pool_malloc(&bar, sizeof(GridBarrier) * nb, s);
  if (e == cudaSuccess) e = pool_malloc(reinterpret_cast<void**>(&rn), sizeof(double) * m * nb, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
  const int64_t sbs = (int64_t)m * n;
  // unit rows first (the sweeps do the same): same row space, better conditioned Gram
  if (e == cudaSuccess) e = row_norms2<T>(S, m, n, n, sbs, rn, s, nb);
  if (e == cudaSuccess) e = scale_rows<T>(S, m, n, sbs, rn, s, nb);
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    e = gemm_f64<T>(m, m, n, nb, S, View::rowmajor(n, sbs), false, S, View::transposed(n, sbs),
                    true, G, View::rowmajor(m, (int64_t)m * m), s);
    if (e == cudaSuccess) e = cholesky_lower<T>(G, m, status, bar, num_sms(), s, nb);
    if (e == cudaSuccess) e = trsm_lower_left<T>(G, S, m, n, status, bar, num_sms(), s, nb);
  }
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (G) cudaFreeAsync(G, s);
  if (status) cudaFreeAsync(status, s);
  if (bar) cudaFreeAsync(bar, s);
  if (rn) cudaFreeAsync(rn, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cbc_cholqr2");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cbc_cholqr2: synchronize");
  if (hs != 0) return fail(hs, "cbc_cholqr2: device status %d", hs);
  return CBC_OK;
}

}  // namespace
}  // namespace cbc

using namespace cbc;

extern "C" {

int cbc_heev(int dtype, int m, int kmax, int nb, void* A, double* lam_out, void* U_out,
             int mixed, void* stream) {
  if (!A || !lam_out || !U_out || m < 1 || kmax < 1 || kmax > m || nb < 1)
    return fail(CBC_ERR_INVALID_ARG, "cbc_heev: bad arguments");
  if (dtype != CBC_F64 && dtype != CBC_C128)
    return fail(CBC_ERR_INVALID_ARG, "cbc_heev: dtype must be CBC_F64 or CBC_C128");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == CBC_C128)
    return heev_t<zdbl>(m, kmax, nb, static_cast<zdbl*>(A), lam_out, static_cast<zdbl*>(U_out),
                        mixed != 0, s);
  return heev_t<double>(m, kmax, nb, static_cast<double*>(A), lam_out, static_cast<double*>(U_out),
                        mixed != 0, s);
}

int cbc_cholqr2(int dtype, int m, int n, int nb, void* S, void* stream) {
  if (!S || m < 1 || n < m || nb < 1)
    return fail(CBC_ERR_INVALID_ARG, "cbc_cholqr2: bad arguments (need 1 <= m <= n)");
  if (dtype != CBC_F64 && dtype != CBC_C128)
    return fail(CBC_ERR_INVALID_ARG, "cbc_cholqr2: dtype must be CBC_F64 or CBC_C128");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == CBC_C128) return cholqr2_t<zdbl>(m, n, nb, static_cast<zdbl*>(S), s);
  return cholqr2_t<double>(m, n, nb, static_cast<double*>(S), s);
}

int cbc_selftest_math(const double* x_dev, double* out_dev, int64_t n, void* stream) {
  if (!x_dev || !out_dev || n < 0) return fail(CBC_ERR_INVALID_ARG, "cbc_selftest_math: bad arguments");
  if (n == 0) return CBC_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int grid = (int)std::min<int64_t>(1024, (n + 255) / 256);
  math_selftest_kernel<<<grid, 256, 0, s>>>(x_dev, out_dev, n);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cbc_selftest_math");
  return CBC_OK;
}

int cbc_selftest_wait(long long limit_cycles, int* returned_out, void* stream) {
  if (limit_cycles < 0 || limit_cycles > 8000000000LL || !returned_out)
    return fail(CBC_ERR_INVALID_ARG, "cbc_selftest_wait: limit must be in [0, 8e9] cycles");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* d = nullptr;  // [0] status, [1] returned, [2] the word nothing writes
  cudaError_t e = pool_malloc(reinterpret_cast<void**>(&d), 4 * sizeof(int), s);
  if (e != cudaSuccess) return cuda_fail(e, "cbc_selftest_wait: alloc");
  int h[2] = {0, 0};
  e = cudaMemsetAsync(d, 0, 4 * sizeof(int), s);
  if (e == cudaSuccess) {
    wait_selftest_kernel<<<1, 32, 0, s>>>(reinterpret_cast<const unsigned int*>(d + 2), d,
                                          limit_cycles, d + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "cbc_selftest_wait");
  if (e2 != cudaSuccess) return cuda_fail(e2, "cbc_selftest_wait: synchronize");
  *returned_out = h[1];
  if (h[0] != 0) return fail(h[0], "cbc_selftest_wait: the wait gave up after %lld cycles",
                             limit_cycles);
  return CBC_OK;
}

}  // extern "C"
