// FP64 Cholesky factorisation and lower-triangular solve for CholeskyQR2.
//
// The backward sweep decomposes S^[i] = R Q^[i] on the leg chi_{i-1} (Eq.
// (tt_cbc_qr_decomp); Eq. (cbc_tree_qr) on trees).  With S of m rows and n >= m columns
// the GPU path forms G = S S^H (FP64 accumulation), factors G = C C^H, and solves
// Q = C^{-1} S; doing it twice (CholeskyQR2) restores orthonormality to FP64 round-off.
// Both kernels are cooperative launches over up to one CTA per SM with 32-wide column
// blocks: a block step is a small factorisation or solve followed by a trailing
// update spread over all CTAs, separated by bounded grid barriers.
#include "kernels.cuh"
#include "planner.h"

namespace cbc {
namespace {

constexpr int NB = 32, TPB = 256;

template <typename T>
__device__ __forceinline__ T ldg_cg(const T* p);
template <>
__device__ __forceinline__ double ldg_cg<double>(const double* p) { return __ldcg(p); }
template <>
__device__ __forceinline__ zdbl ldg_cg<zdbl>(const zdbl* p) {
  double2 v = __ldcg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

template <typename T>
struct CholArgs {
  T* G;
  int m;
  int* status;
  GridBarrier* bar;
};

// G (row-major m x m, Hermitian, lower triangle read) -> C (lower triangle), G = C C^H
template <typename T>
__global__ void __launch_bounds__(TPB) chol_kernel(CholArgs<T> a) {
  using O = ops<T>;
  __shared__ T blk[NB][NB + 1];
  __shared__ int s_bad;
  const int m = a.m, P = gridDim.x, cta = blockIdx.x;
  const int gtid = cta * blockDim.x + threadIdx.x, gthreads = P * blockDim.x;
  for (int b0 = 0; b0 < m; b0 += NB) {
    const int nb = min(NB, m - b0);
    // (1) diagonal block on CTA 0
    if (cta == 0) {
      for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
        int i = t / nb, l = t % nb;
        blk[i][l] = (l <= i) ? ldg_cg(a.G + (int64_t)(b0 + i) * m + b0 + l) : O::zero();
      }
      if (threadIdx.x == 0) s_bad = 0;
      __syncthreads();
      for (int jj = 0; jj < nb; ++jj) {
        double piv = O::real(blk[jj][jj]);
        if (!(piv > 0.0) || !isfinite(piv)) {
          if (threadIdx.x == 0) s_bad = 1;
          break;
        }
        double c = sqrt(piv);
        __syncthreads();
        if (threadIdx.x == 0) blk[jj][jj] = O::make(c, 0.0);
        for (int i = jj + 1 + threadIdx.x; i < nb; i += blockDim.x)
          blk[i][jj] = O::scale(1.0 / c, blk[i][jj]);
        __syncthreads();
        for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
          int i = t / nb, l = t % nb;
          if (i > jj && l > jj && l <= i) blk[i][l] = blk[i][l] - blk[i][jj] * O::conj(blk[l][jj]);
        }
        __syncthreads();
      }
      __syncthreads();
      if (s_bad) {
        if (threadIdx.x == 0) set_status(a.status, CBC_ERR_NOT_POSITIVE_DEFINITE);
      } else {
        for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
          int i = t / nb, l = t % nb;
          if (l <= i) a.G[(int64_t)(b0 + i) * m + b0 + l] = blk[i][l];
        }
      }
      __threadfence();
    }
    if (!grid_sync(a.bar, a.status)) return;
    if (*((volatile int*)a.status) != 0) return;
    // (2) panel rows below: X = G[r, blk] C_bb^{-H}, one thread per row
    for (int r = b0 + nb + gtid; r < m; r += gthreads) {
      T* row = a.G + (int64_t)r * m + b0;
      T x[NB];
      for (int l = 0; l < nb; ++l) {
        T s = ldg_cg(row + l);
        for (int t = 0; t < l; ++t)
          s = s - x[t] * O::conj(ldg_cg(a.G + (int64_t)(b0 + l) * m + b0 + t));
        double dl = O::real(ldg_cg(a.G + (int64_t)(b0 + l) * m + b0 + l));
        x[l] = O::scale(1.0 / dl, s);
      }
      for (int l = 0; l < nb; ++l) row[l] = x[l];
    }
    if (!grid_sync(a.bar, a.status)) return;
    // (3) trailing update of the lower triangle: G[r][c] -= sum_t X[r][t] conj(X[c][t])
    const int r0 = b0 + nb;
    const int64_t nt = (int64_t)(m - r0) * (m - r0);
    for (int64_t t = gtid; t < nt; t += gthreads) {
      int r = r0 + (int)(t / (m - r0)), c = r0 + (int)(t % (m - r0));
      if (c > r) continue;
      const T* xr = a.G + (int64_t)r * m + b0;
      const T* xc = a.G + (int64_t)c * m + b0;
      T s = O::zero();
      for (int l = 0; l < nb; ++l) s = O::fma(ldg_cg(xr + l), O::conj(ldg_cg(xc + l)), s);
      T* g = a.G + (int64_t)r * m + c;
      *g = ldg_cg(g) - s;
    }
    if (!grid_sync(a.bar, a.status)) return;
  }
}

template <typename T>
struct TrsmArgs {
  const T* C;
  T* S;
  int m, n;
  int* status;
  GridBarrier* bar;
};

// S (m x n) <- C^{-1} S with C lower triangular (m x m)
template <typename T>
__global__ void __launch_bounds__(TPB) trsm_kernel(TrsmArgs<T> a) {
  using O = ops<T>;
  const int m = a.m, n = a.n, P = gridDim.x;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, gthreads = P * blockDim.x;
  for (int b0 = 0; b0 < m; b0 += NB) {
    const int nb = min(NB, m - b0);
    // (1) diagonal block solve, one thread per column
    for (int c = gtid; c < n; c += gthreads) {
      T x[NB];
      for (int l = 0; l < nb; ++l) {
        T s = ldg_cg(a.S + (int64_t)(b0 + l) * n + c);
        const T* crow = a.C + (int64_t)(b0 + l) * m + b0;
        for (int t = 0; t < l; ++t) s = s - crow[t] * x[t];
        x[l] = O::scale(1.0 / O::real(crow[l]), s);
      }
      for (int l = 0; l < nb; ++l) a.S[(int64_t)(b0 + l) * n + c] = x[l];
    }
    if (!grid_sync(a.bar, a.status)) return;
    // (2) update of the rows below
    const int r0 = b0 + nb;
    const int64_t nt = (int64_t)(m - r0) * n;
    for (int64_t t = gtid; t < nt; t += gthreads) {
      int r = r0 + (int)(t / n), c = (int)(t % n);
      const T* crow = a.C + (int64_t)r * m + b0;
      T s = O::zero();
      for (int l = 0; l < nb; ++l) s = O::fma(crow[l], ldg_cg(a.S + (int64_t)(b0 + l) * n + c), s);
      T* dst = a.S + (int64_t)r * n + c;
      *dst = ldg_cg(dst) - s;
    }
    if (!grid_sync(a.bar, a.status)) return;
  }
}

}  // namespace

template <typename T>
cudaError_t cholesky_lower(T* G, int m, int* status, void* bar, int num_sms, cudaStream_t s) {
  // FP64 is scarce per SM on this part: spread the trailing updates over many SMs
  int P = max(1, min(num_sms, (m * m) / 128));
  cudaError_t err = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
  if (err != cudaSuccess) return err;
  note_launches(CBC_K_CHOLQR, 1);
  CholArgs<T> a{G, m, status, (GridBarrier*)bar};
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)chol_kernel<T>, dim3(P), dim3(TPB), args, 0, s);
}

template <typename T>
cudaError_t trsm_lower_left(const T* C, T* S, int m, int n, int* status, void* bar, int num_sms,
                            cudaStream_t s) {
  int64_t pw = ((int64_t)m * n) / 256;
  int P = (int)(pw < 1 ? 1 : (pw > num_sms ? num_sms : pw));
  cudaError_t err = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s);
  if (err != cudaSuccess) return err;
  note_launches(CBC_K_CHOLQR, 1);
  TrsmArgs<T> a{C, S, m, n, status, (GridBarrier*)bar};
  void* args[] = {&a};
  return cudaLaunchCooperativeKernel((const void*)trsm_kernel<T>, dim3(P), dim3(TPB), args, 0, s);
}

template cudaError_t cholesky_lower<double>(double*, int, int*, void*, int, cudaStream_t);
template cudaError_t cholesky_lower<zdbl>(zdbl*, int, int*, void*, int, cudaStream_t);
template cudaError_t trsm_lower_left<double>(const double*, double*, int, int, int*, void*, int,
                                             cudaStream_t);
template cudaError_t trsm_lower_left<zdbl>(const zdbl*, zdbl*, int, int, int*, void*, int,
                                           cudaStream_t);

}  // namespace cbc
