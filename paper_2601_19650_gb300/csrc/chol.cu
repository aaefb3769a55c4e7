// FP64 Cholesky factorisation and lower-triangular solve for CholeskyQR2.
//
// The backward sweep decomposes S^[i] = R Q^[i] on the leg chi_{i-1} (Eq.
// (tt_cbc_qr_decomp); Eq. (cbc_tree_qr) on trees).  With S of m rows and n >= m columns
// the GPU path forms G = S S^H, factors G = C C^H, and solves Q = C^{-1} S; doing it
// twice (CholeskyQR2) restores orthonormality to FP64 round-off.
//
// Cholesky: one group of CTAs that wait on each other (a thread-block cluster of up to
// 16 CTAs, else a cooperative launch), 32-wide column blocks.  Per block, CTA 0 factors
// the diagonal block in shared memory, every other row of the panel is solved by one
// warp (shuffles carry the solved entries), and the trailing lower triangle is updated
// from a shared-memory copy of the panel; bounded grid barriers separate the phases.
// Triangular solve: columns of S are independent, so each warp owns one column and runs
// the forward substitution in 32-row groups without any inter-CTA synchronisation.
// Divisions use Newton reciprocals (rcp64): long dependent chains of FP64 divisions are
// slow on this part.
#include <algorithm>

#include "df.cuh"
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
__device__ __forceinline__ T shfl(T v, int src);
template <>
__device__ __forceinline__ double shfl<double>(double v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
template <>
__device__ __forceinline__ zdbl shfl<zdbl>(zdbl v, int src) {
  return {__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}

template <typename T>
struct CholArgs {
  T* G;
  int m;
  int* status;
  GridBarrier* bar;
  int P;  // CTAs per matrix; CTA b works on matrix b / P (G + (b / P) m^2, bar + b / P)
};

// G (row-major m x m, Hermitian, lower triangle read) -> C (lower triangle), G = C C^H
// PSMEM: the panel of the trailing update is copied to shared memory (m up to ~440
// complex); else the update reads it from global memory (L2).
template <typename T, bool PSMEM>
__global__ void __launch_bounds__(TPB) chol_kernel(CholArgs<T> a) {
  using O = ops<T>;
  extern __shared__ unsigned char sm_raw[];
  T* pan = reinterpret_cast<T*>(sm_raw);  // panel rows [b0, m) x NB, or the diag block
  __shared__ double s_rd[NB];             // reciprocals of the diagonal of the block
  __shared__ int s_bad;
  const int m = a.m, P = a.P, cta = blockIdx.x % P;
  a.G += (int64_t)(blockIdx.x / P) * m * m;
  a.bar += blockIdx.x / P;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int b0 = 0; b0 < m; b0 += NB) {
    const int nb = min(NB, m - b0);
    // (1) diagonal block on CTA 0
    if (cta == 0) {
      T* blk = pan;  // nb x NB
      for (int t = threadIdx.x; t < nb * NB; t += blockDim.x) {
        int i = t / NB, l = t % NB;
        blk[t] = (l <= i && l < nb) ? ldg_cg(a.G + (int64_t)(b0 + i) * m + b0 + l) : O::zero();
      }
      if (threadIdx.x == 0) s_bad = 0;
      __syncthreads();
      for (int jj = 0; jj < nb; ++jj) {
        const double piv = O::real(blk[jj * NB + jj]);
        if (!(piv > 0.0) || !isfinite(piv)) {
          if (threadIdx.x == 0) s_bad = 1;
          break;
        }
        const double rc = rsqrt64(piv);  // 1 / sqrt(piv)
        const double rp = rc * rc;        // 1 / piv
        // trailing update with the unscaled column (divide by piv), then scale column
        for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
          int i = t / nb, l = t % nb;
          if (i > jj && l > jj && l <= i)
            blk[i * NB + l] = blk[i * NB + l] -
                              O::scale(rp, blk[i * NB + jj] * O::conj(blk[l * NB + jj]));
        }
        __syncthreads();
        for (int i = jj + threadIdx.x; i < nb; i += blockDim.x)
          blk[i * NB + jj] = (i == jj) ? O::make(piv * rc, 0.0) : O::scale(rc, blk[i * NB + jj]);
        __syncthreads();
      }
      __syncthreads();
      if (s_bad) {
        if (threadIdx.x == 0) set_status(a.status, CBC_ERR_NOT_POSITIVE_DEFINITE);
      } else {
        for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
          int i = t / nb, l = t % nb;
          if (l <= i) a.G[(int64_t)(b0 + i) * m + b0 + l] = blk[i * NB + l];
        }
      }
      __threadfence();
    }
    if (!grid_sync(a.bar, a.status, (unsigned)P)) return;
    if (*((volatile int*)a.status) != 0) return;
    // (2) panel rows below: x C_bb^H = g, one warp per row (lane l holds entry l)
    {
      T* cbb = pan;  // nb x NB copy of the factored block
      for (int t = threadIdx.x; t < nb * NB; t += blockDim.x) {
        int i = t / NB, l = t % NB;
        cbb[t] = (l <= i && l < nb) ? ldg_cg(a.G + (int64_t)(b0 + i) * m + b0 + l) : O::zero();
      }
      for (int i = threadIdx.x; i < nb; i += blockDim.x)
        s_rd[i] = rcp64(O::real(ldg_cg(a.G + (int64_t)(b0 + i) * m + b0 + i)));
      __syncthreads();
      for (int r = b0 + nb + cta * nw + warp; r < m; r += P * nw) {
        T* row = a.G + (int64_t)r * m + b0;
        T acc = (lane < nb) ? ldg_cg(row + lane) : O::zero();
        T x = O::zero();
        for (int t = 0; t < nb; ++t) {
          const T xt = shfl(O::scale(s_rd[t], acc), t);  // lane t is final at step t
          if (lane == t) x = xt;
          if (lane > t && lane < nb) acc = acc - xt * O::conj(cbb[lane * NB + t]);
        }
        if (lane < nb) row[lane] = x;
      }
    }
    if (!grid_sync(a.bar, a.status, (unsigned)P)) return;
    // (3) trailing update of the lower triangle from a shared copy of the panel
    const int r0 = b0 + nb;
    if (r0 < m) {
      const int rows = m - r0;
      if (PSMEM) {
        for (int t = threadIdx.x; t < rows * NB; t += blockDim.x) {
          int i = t / NB, l = t % NB;
          pan[t] = (l < nb) ? ldg_cg(a.G + (int64_t)(r0 + i) * m + b0 + l) : O::zero();
        }
        __syncthreads();
      }
      const int64_t nt = (int64_t)rows * (rows + 1) / 2;
      for (int64_t t = (int64_t)cta * blockDim.x + threadIdx.x; t < nt; t += (int64_t)P * blockDim.x) {
        // t -> (i, c) with c <= i in the packed lower triangle
        const int i = tri_row(t);
        const int c = (int)(t - (int64_t)i * (i + 1) / 2);
        T sacc = O::zero();
        if (PSMEM) {
#pragma unroll 8
          for (int l = 0; l < NB; ++l) sacc = O::fma(pan[i * NB + l], O::conj(pan[c * NB + l]), sacc);
        } else {
          const T* pi = a.G + (int64_t)(r0 + i) * m + b0;
          const T* pc = a.G + (int64_t)(r0 + c) * m + b0;
          for (int l = 0; l < nb; ++l) sacc = O::fma(ldg_cg(pi + l), O::conj(ldg_cg(pc + l)), sacc);
        }
        T* g = a.G + (int64_t)(r0 + i) * m + r0 + c;
        *g = ldg_cg(g) - sacc;
      }
    }
    if (!grid_sync(a.bar, a.status, (unsigned)P)) return;
  }
}

// One CTA per matrix of a batch (blockIdx.x), the lower triangle packed in shared memory
// ((i, l) at i (i + 1) / 2 + l): right-looking, one column per step, no grid barriers.
// For batches, where the matrices themselves fill the SMs.
template <typename T>
__global__ void __launch_bounds__(TPB) chol1_kernel(T* G, int m, int* status) {
  using O = ops<T>;
  extern __shared__ unsigned char sm_raw[];
  T* L = reinterpret_cast<T*>(sm_raw);
  __shared__ double s_rc;
  __shared__ int s_bad;
  G += (int64_t)blockIdx.x * m * m;
  const int64_t tri = (int64_t)m * (m + 1) / 2;
  for (int64_t t = threadIdx.x; t < tri; t += blockDim.x) {
    const int i = tri_row(t);
    L[t] = G[(int64_t)i * m + (t - (int64_t)i * (i + 1) / 2)];
  }
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    const int64_t dj = (int64_t)j * (j + 1) / 2 + j;
    if (threadIdx.x == 0) {
      const double piv = O::real(L[dj]);
      if (!(piv > 0.0) || !isfinite(piv)) {
        s_bad = 1;
      } else {
        const double rc = rsqrt64(piv);  // 1 / sqrt(piv)
        L[dj] = O::make(piv * rc, 0.0);
        s_rc = rc;
      }
    }
    __syncthreads();
    if (s_bad) break;
    const double rc = s_rc;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
      T* x = L + (int64_t)i * (i + 1) / 2 + j;
      *x = O::scale(rc, *x);
    }
    __syncthreads();
    // trailing lower triangle (i, l), j < l <= i: L[i][l] -= L[i][j] conj(L[l][j])
    const int r = m - j - 1;
    const int64_t nt = (int64_t)r * (r + 1) / 2;
    for (int64_t t = threadIdx.x; t < nt; t += blockDim.x) {
      const int ii = tri_row(t);
      const int i = j + 1 + ii, l = j + 1 + (int)(t - (int64_t)ii * (ii + 1) / 2);
      const int64_t bi = (int64_t)i * (i + 1) / 2, bl = (int64_t)l * (l + 1) / 2;
      L[bi + l] = O::fma(O::scale(-1.0, L[bi + j]), O::conj(L[bl + j]), L[bi + l]);
    }
    __syncthreads();
  }
  if (s_bad) {
    if (threadIdx.x == 0) set_status(status, CBC_ERR_NOT_POSITIVE_DEFINITE);
    return;
  }
  for (int64_t t = threadIdx.x; t < tri; t += blockDim.x) {
    const int i = tri_row(t);
    G[(int64_t)i * m + (t - (int64_t)i * (i + 1) / 2)] = L[t];
  }
}

// S (m x n) <- C^{-1} S, C lower triangular (row-major m x m).  One warp per column.
template <typename T, bool CSMEM>
__global__ void trsm_cols_kernel(const T* C, T* S, int m, int n) {
  using O = ops<T>;
  C += (int64_t)blockIdx.y * m * m;  // problem blockIdx.y of a batch
  S += (int64_t)blockIdx.y * m * n;
  extern __shared__ unsigned char sm_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T* cl = reinterpret_cast<T*>(sm_raw);  // packed lower triangle (CSMEM)
  double* rd = reinterpret_cast<double*>(cl + (CSMEM ? (size_t)m * (m + 1) / 2 : 0));
  T* xs = reinterpret_cast<T*>(rd + m);
  if (CSMEM) {
    const int64_t tot = (int64_t)m * (m + 1) / 2;
    for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
      const int i = tri_row(t);
      const int l = (int)(t - (int64_t)i * (i + 1) / 2);
      cl[t] = C[(int64_t)i * m + l];
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) rd[i] = rcp64(O::real(C[(int64_t)i * m + i]));
  __syncthreads();
  const int c = blockIdx.x * nw + warp;
  if (c >= n) return;
  T* x = xs + (size_t)warp * m;
  auto cel = [&](int i, int l) -> T {
    return CSMEM ? cl[(int64_t)i * (i + 1) / 2 + l] : C[(int64_t)i * m + l];
  };
  for (int b0 = 0; b0 < m; b0 += 32) {
    const int i = b0 + lane;
    const bool live = i < m;
    T acc = live ? S[(int64_t)i * n + c] : O::zero();
    for (int l = 0; l < b0; ++l) acc = acc - (live ? cel(i, l) : O::zero()) * x[l];
    const int gb = min(32, m - b0);
    for (int t = 0; t < gb; ++t) {
      const T xt = shfl(O::scale(rd[b0 + t], acc), t);
      if (lane == t) x[i] = xt;
      if (lane > t && live) acc = acc - cel(i, b0 + t) * xt;
    }
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) S[(int64_t)i * n + c] = x[i];
}

// The same solve in double-float arithmetic (the mixed path): the factor's lower
// triangle D and the reciprocal pivots R come as double-float pairs (converted once per
// solve by to_df_kernel), and the accumulation and the solution stay double-float; FP64
// only to read S and to write the result.
template <typename T, bool CSMEM>
__global__ void trsm_cols_df_kernel(const typename dfof<T>::type* D, const df1* R, T* S, int m,
                                    int n) {
  using O = ops<T>;
  using E = typename dfof<T>::type;
  D += (int64_t)blockIdx.y * m * m;
  R += (int64_t)blockIdx.y * m;
  S += (int64_t)blockIdx.y * m * n;
  extern __shared__ unsigned char sm_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  E* cl = reinterpret_cast<E*>(sm_raw);  // packed lower triangle (CSMEM)
  df1* rd = reinterpret_cast<df1*>(cl + (CSMEM ? (size_t)m * (m + 1) / 2 : 0));
  E* xs = reinterpret_cast<E*>(rd + m);
  if (CSMEM) {
    const int64_t tot = (int64_t)m * (m + 1) / 2;
    for (int64_t t = threadIdx.x; t < tot; t += blockDim.x) {
      const int i = tri_row(t);
      cl[t] = D[(int64_t)i * m + (int)(t - (int64_t)i * (i + 1) / 2)];
    }
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) rd[i] = R[i];
  __syncthreads();
  const int c = blockIdx.x * nw + warp;
  if (c >= n) return;
  E* x = xs + (size_t)warp * m;
  auto cel = [&](int i, int l) -> E {
    return CSMEM ? cl[(int64_t)i * (i + 1) / 2 + l] : D[(int64_t)i * m + l];
  };
  const df1 z1{0.f, 0.f};
  for (int b0 = 0; b0 < m; b0 += 32) {
    const int i = b0 + lane;
    const bool live = i < m;
    E acc = live ? to_df(S[(int64_t)i * n + c]) : E{};
    if (live)
      for (int l = 0; l < b0; ++l) acc = dff(df_neg(cel(i, l)), x[l], acc);
    const int gb = min(32, m - b0);
    for (int t = 0; t < gb; ++t) {
      E xt;
      if constexpr (O::cplx)
        xt = E{df_fma(acc.re, rd[b0 + t], z1), df_fma(acc.im, rd[b0 + t], z1)};
      else
        xt = df_fma(acc, rd[b0 + t], z1);
      xt = df_shfl_idx(xt, t);
      if (lane == t) x[i] = xt;
      if (lane > t && live) acc = dff(df_neg(cel(i, b0 + t)), xt, acc);
    }
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) S[(int64_t)i * n + c] = from_df(x[i]);
}

// The lower triangle of C (row-major m x m) and the reciprocals of its (real) pivots as
// double-float pairs, for trsm_cols_df_kernel; nb factors, m*m (and m) elements apart.
template <typename T>
__global__ void to_df_kernel(const T* C, typename dfof<T>::type* D, df1* R, int m) {
  using O = ops<T>;
  C += (int64_t)blockIdx.y * m * m;
  D += (int64_t)blockIdx.y * m * m;
  R += (int64_t)blockIdx.y * m;
  const int64_t tot = (int64_t)m * m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / m), l = (int)(t % m);
    if (l <= i) D[t] = to_df(C[t]);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    R[i] = df_make(rcp64(O::real(C[(int64_t)i * m + i])));
}

}  // namespace

template <typename T>
cudaError_t cholesky_lower(T* G, int m, int* status, void* bar, int num_sms, cudaStream_t s,
                           int nb) {
  // FP64 is scarce per SM on this part: spread the trailing updates over several SMs,
  // one cluster of up to 16 CTAs per matrix when it fits (concurrent with other
  // streams' work), else a cooperative launch over more SMs per matrix
  cudaError_t err = cudaMemsetAsync(bar, 0, sizeof(GridBarrier) * nb, s);
  if (err != cudaSuccess) return err;
  // the panel in shared memory when it fits, else read from global memory
  const bool psmem = (size_t)std::max(m, NB) * NB * sizeof(T) <= 200 * 1024;
  const size_t shm = (size_t)(psmem ? std::max(m, NB) : NB) * NB * sizeof(T);
  const void* kch = psmem ? (const void*)chol_kernel<T, true> : (const void*)chol_kernel<T, false>;
  if (shm > 48 * 1024) {
    err = allow_max_smem(kch);
    if (err != cudaSuccess) return err;
  }
  note_launches(CBC_K_CHOLQR, 1);
  // a batch of 8 or more: one CTA per matrix (its FP64 work spread over the batch
  // instead of over a cluster per matrix)
  const size_t tri_bytes = (size_t)m * (m + 1) / 2 * sizeof(T);
  if (nb >= 8 && tri_bytes <= 200 * 1024) {
    err = allow_max_smem((const void*)chol1_kernel<T>);
    if (err != cudaSuccess) return err;
    chol1_kernel<T><<<nb, TPB, tri_bytes, s>>>(G, m, status);
    return cudaGetLastError();
  }
  int P = std::max(1, std::min(16, (m * m) / 256));
  if (cluster_ctas(kch, P, TPB, shm) == P) {
    CholArgs<T> a{G, m, status, (GridBarrier*)bar, P};
    void* args[] = {&a};
    return launch_cluster(kch, P, nb * P, TPB, shm, args, s);
  }
  P = std::max(1, std::min(num_sms, (m * m) / 256));
  for (int b = 0; b < nb; ++b) {
    CholArgs<T> a{G + (int64_t)b * m * m, m, status, (GridBarrier*)bar + b, P};
    void* args[] = {&a};
    err = cudaLaunchCooperativeKernel(kch, dim3(P), dim3(TPB), args, shm, s);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t trsm_lower_left(const T* C, T* S, int m, int n, int* status, void* bar, int num_sms,
                            cudaStream_t s, int nb, void* dfbuf) {
  (void)status;
  (void)bar;
  (void)num_sms;
  if (dfbuf) {  // double-float solve: the factor converted once, then one warp per column
    using E = typename dfof<T>::type;
    E* D = static_cast<E*>(dfbuf);
    df1* R = reinterpret_cast<df1*>(D + (size_t)nb * m * m);
    note_launches(CBC_K_CHOLQR, 2);
    to_df_kernel<T><<<dim3(std::max(1, std::min(64, (m * m + 255) / 256)), nb), 256, 0, s>>>(C, D, R, m);
    const int nw = nb >= 8 ? 8 : 4;
    const size_t tri = (size_t)m * (m + 1) / 2 * sizeof(E);
    const size_t rest = (size_t)m * sizeof(df1) + (size_t)nw * m * sizeof(E);
    const dim3 grid((n + nw - 1) / nw, nb);
    cudaError_t err;
    if (tri + rest <= 200 * 1024) {
      err = allow_max_smem((const void*)trsm_cols_df_kernel<T, true>);
      if (err != cudaSuccess) return err;
      trsm_cols_df_kernel<T, true><<<grid, 32 * nw, tri + rest, s>>>(D, R, S, m, n);
    } else {
      if (rest > 48 * 1024) {
        err = allow_max_smem((const void*)trsm_cols_df_kernel<T, false>);
        if (err != cudaSuccess) return err;
      }
      trsm_cols_df_kernel<T, false><<<grid, 32 * nw, rest, s>>>(D, R, S, m, n);
    }
    return cudaGetLastError();
  }
  // warps (columns) per CTA sharing one staged triangle: two per SM sub-partition when a
  // batch provides the CTAs, else one (more CTAs for a lone solve)
  const int nw = nb >= 8 ? 8 : 4;
  const size_t tri = (size_t)m * (m + 1) / 2 * sizeof(T);
  const size_t rest = (size_t)m * sizeof(double) + (size_t)nw * m * sizeof(T);
  note_launches(CBC_K_CHOLQR, 1);
  const dim3 grid((n + nw - 1) / nw, nb);
  cudaError_t err;
  if (tri + rest <= 200 * 1024) {
    err = allow_max_smem((const void*)trsm_cols_kernel<T, true>);
    if (err != cudaSuccess) return err;
    trsm_cols_kernel<T, true><<<grid, 32 * nw, tri + rest, s>>>(C, S, m, n);
  } else {
    if (rest > 48 * 1024) {
      err = allow_max_smem((const void*)trsm_cols_kernel<T, false>);
      if (err != cudaSuccess) return err;
    }
    trsm_cols_kernel<T, false><<<grid, 32 * nw, rest, s>>>(C, S, m, n);
  }
  return cudaGetLastError();
}

template cudaError_t cholesky_lower<double>(double*, int, int*, void*, int, cudaStream_t, int);
template cudaError_t cholesky_lower<zdbl>(zdbl*, int, int*, void*, int, cudaStream_t, int);
template cudaError_t trsm_lower_left<double>(const double*, double*, int, int, int*, void*, int,
                                             cudaStream_t, int, void*);
template cudaError_t trsm_lower_left<zdbl>(const zdbl*, zdbl*, int, int, int*, void*, int,
                                           cudaStream_t, int, void*);

}  // namespace cbc
