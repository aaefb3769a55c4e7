// Small element-wise kernels of the CBC pipeline: dtype widening / narrowing, the
// per-step renormalisation with a running log scale, the m > n truncation factor
// diag(sqrt(lambda)) V^H, and identity fill for the trivial LQ case.
#include <algorithm>
#include <mutex>
#include <vector>

#include "kernels.cuh"
#include "planner.h"

namespace cbc {
namespace {

// batched kernels: problem blockIdx.y, its data n (or k x n) elements apart
template <typename T>
__global__ void sumsq_kernel(const T* x, int64_t n, double* out) {
  x += (int64_t)blockIdx.y * n;
  out += blockIdx.y;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += ops<T>::abs2(x[i]);
  s = warp_sum(s);
  __shared__ double sh[32];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = s;
  __syncthreads();
  if (w == 0) {
    s = (lane < (blockDim.x >> 5)) ? sh[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) atomicAdd(out, s);
  }
}

template <typename T>
__global__ void scale_kernel(T* x, int64_t n, const double* sumsq, double* log_acc, int* status,
                             int shared_log) {
  x += (int64_t)blockIdx.y * n;
  sumsq += blockIdx.y;
  if (!shared_log) log_acc += blockIdx.y;
  double ss = *sumsq;
  bool ok = isfinite(ss) && ss > 0.0;
  if (!ok) {  // NaN / Inf, or an all-zero tensor (then O|psi> itself vanishes)
    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(status, CBC_ERR_NUMERICAL);
    return;
  }
  double inv = rsqrt(ss);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (shared_log)
      atomicAdd(log_acc, 0.5 * log(ss));
    else
      *log_acc += 0.5 * log(ss);
  }
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = ops<T>::scale(inv, x[i]);
}

template <typename T>
__global__ void scaled_adjoint_kernel(const T* V, int ldv, const double* lam, const int* k_dev,
                                      int n, T* L, int64_t l_bs) {
  V += (int64_t)blockIdx.y * n * ldv;
  lam += (int64_t)blockIdx.y * n;
  k_dev += blockIdx.y;
  L += (int64_t)blockIdx.y * l_bs;
  int k = *k_dev;
  int64_t total = (int64_t)k * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(t / n), c = (int)(t % n);
    double sl = sqrt(fmax(lam[r], 0.0));
    L[t] = ops<T>::scale(sl, ops<T>::conj(V[(int64_t)c * ldv + r]));
  }
}

// between nb separate tensors (ptrs[b], n elements each) and one buffer holding them
// `stride` elements apart; instance blockIdx.y
template <typename T>
__global__ void group_copy_kernel(T* const* ptrs, T* buf, int64_t stride, int64_t n, int to_group) {
  T* p = ptrs[blockIdx.y];
  T* g = buf + (int64_t)blockIdx.y * stride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (to_group)
      g[i] = p[i];
    else
      p[i] = g[i];
  }
}

template <typename T>
__global__ void identity_kernel(T* dst, int n) {
  dst += (int64_t)blockIdx.y * n * n;
  int64_t total = (int64_t)n * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int r = (int)(t / n), c = (int)(t % n);
    dst[t] = (r == c) ? ops<T>::one() : ops<T>::zero();
  }
}

__global__ void widen_kernel(const void* src, int dt, double* dst, int64_t n_scalar,
                             int* nonfinite) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_scalar;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v;
    if (dt == CBC_F32 || dt == CBC_C64)
      v = (double)static_cast<const float*>(src)[i];
    else
      v = static_cast<const double*>(src)[i];
    bad = bad || !isfinite(v);
    dst[i] = v;
  }
  if (nonfinite && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) *nonfinite = 1;
}

__global__ void narrow_kernel(const double* src, void* dst, int dt, int64_t n_scalar) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_scalar;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (dt == CBC_F32 || dt == CBC_C64)
      static_cast<float*>(dst)[i] = (float)src[i];
    else
      static_cast<double*>(dst)[i] = src[i];
  }
}

struct PermArgs {
  int rank;
  int64_t out_dims[8];
  int64_t in_stride_of_out[8];  // stride in `in` of each output axis
};

template <typename T>
__global__ void permute_kernel(const T* in, T* out, int64_t total, PermArgs a) {
  in += (int64_t)blockIdx.y * total;  // tensor blockIdx.y of a batch
  out += (int64_t)blockIdx.y * total;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = t, off = 0;
    for (int d = a.rank - 1; d >= 0; --d) {
      const int64_t i = rem % a.out_dims[d];
      rem /= a.out_dims[d];
      off += i * a.in_stride_of_out[d];
    }
    out[t] = in[off];
  }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(4096, (n + 255) / 256)); }

// one warp per row; problem blockIdx.y
template <typename T>
__global__ void row_norms2_kernel(const T* W, int rows, int cols, int64_t ld, int64_t bs,
                                  double* out) {
  W += (int64_t)blockIdx.y * bs;
  out += (int64_t)blockIdx.y * rows;
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += nw) {
    const T* row = W + (int64_t)r * ld;
    double acc = 0.0;
    for (int c = lane; c < cols; c += 32) acc += ops<T>::abs2(row[c]);
    acc = warp_sum(acc);
    if (lane == 0) out[r] = acc;
  }
}

// columns on threadIdx.x (32 per CTA, coalesced), rows split over threadIdx.y and the
// CTAs of blockIdx.x's row chunks; partial sums added into out (zeroed before)
template <typename T>
__global__ void col_norms2_kernel(const T* W, int rows, int cols, int64_t ld, int64_t bs,
                                  int rows_per_cta, double* out) {
  W += (int64_t)blockIdx.y * bs;
  out += (int64_t)blockIdx.y * cols;
  __shared__ double part[8][33];
  const int r0 = blockIdx.x * rows_per_cta, r1 = min(rows, r0 + rows_per_cta);
  for (int c0 = 0; c0 < cols; c0 += 32) {
    const int c = c0 + threadIdx.x;
    double acc = 0.0;
    if (c < cols)
      for (int r = r0 + threadIdx.y; r < r1; r += blockDim.y) acc += ops<T>::abs2(W[(int64_t)r * ld + c]);
    part[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && c < cols) {
      double t = 0.0;
      for (int q = 0; q < (int)blockDim.y; ++q) t += part[q][threadIdx.x];
      atomicAdd(out + c, t);
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void diff_sumsq_kernel(const T* A, int64_t a_bs, const T* B, T* C, int64_t n,
                                  double* out) {
  A += (int64_t)blockIdx.y * a_bs;
  B += (int64_t)blockIdx.y * n;
  if (C) C += (int64_t)blockIdx.y * n;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T d = A[i] - B[i];
    if (C) C[i] = d;
    acc += ops<T>::abs2(d);
  }
  acc = warp_sum(acc);
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = acc;
  __syncthreads();
  if (w == 0) {
    acc = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    acc = warp_sum(acc);
    if (lane == 0) atomicAdd(out + blockIdx.y, acc);
  }
}

template <typename T>
__global__ void scaled_adjoint_w_kernel(const T* V, int ldv, const double* w, int64_t w_bs, int k,
                                        int n, T* L, int64_t l_bs) {
  V += (int64_t)blockIdx.y * n * ldv;
  w += (int64_t)blockIdx.y * w_bs;
  L += (int64_t)blockIdx.y * l_bs;
  const int64_t total = (int64_t)k * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / n), c = (int)(t % n);
    L[t] = ops<T>::scale(sqrt(fmax(w[r], 0.0)), ops<T>::conj(V[(int64_t)c * ldv + r]));
  }
}

template <typename T>
__global__ void scale_rows_kernel(T* X, int rows, int cols, int64_t bs, const double* norms2) {
  X += (int64_t)blockIdx.y * bs;
  norms2 += (int64_t)blockIdx.y * rows;
  const int64_t total = (int64_t)rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double nr = norms2[t / cols];
    if (nr > 0.0) X[t] = ops<T>::scale(rsqrt(nr), X[t]);
  }
}

// out[b] = sum_i Re G_b[i, i] (G_b g x g, bs elements apart): one CTA per matrix
template <typename T>
__global__ void trace_kernel(const T* G, int g, int64_t bs, double* out) {
  __shared__ double red[256];
  G += (int64_t)blockIdx.x * bs;
  double acc = 0.0;
  for (int i = threadIdx.x; i < g; i += blockDim.x) acc += ops<T>::real(G[(int64_t)i * g + i]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// out[c, r] = conj(in[r, c]) (in: rows x cols, out: cols x rows, both row-major)
template <typename T>
__global__ void adjoint_kernel(const T* in, int rows, int cols, T* out) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / cols, c = t % cols;
    out[c * rows + r] = ops<T>::conj(in[t]);
  }
}

// G_b[i, i] += shift (real) for i < m, nb matrices m*m elements apart
template <typename T>
__global__ void add_diag_kernel(T* G, int m, double shift) {
  G += (int64_t)blockIdx.y * m * m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    T v = G[(int64_t)i * m + i];
    G[(int64_t)i * m + i] = ops<T>::make(ops<T>::real(v) + shift, ops<T>::imag(v));
  }
}

template <typename T>
__global__ void copy_batched_kernel(const T* src, int64_t s_bs, T* dst, int64_t d_bs, int64_t n) {
  src += (int64_t)blockIdx.y * s_bs;
  dst += (int64_t)blockIdx.y * d_bs;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

}  // namespace

cudaError_t allow_max_smem(const void* func) {
  // once per kernel: the attribute call takes a driver lock and costs microseconds, and
  // the planners ask before many launches
  static std::mutex mu;
  static std::vector<const void*> done;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const void* f : done)
      if (f == func) return cudaSuccess;
  }
  static int optin = 0;
  if (optin == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    optin = v > 0 ? v : 48 * 1024;
  }
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(mu);
    done.push_back(func);
  }
  return e;
}

// Largest cluster size <= want (at most 16) for which one cluster of `func` with this
// block and shared-memory size fits on the GPU; 0 if none.  Cached per (func, smem).
int cluster_ctas(const void* func, int want, int threads, size_t smem) {
  struct Entry {
    const void* f;
    size_t smem;
    int threads, want, got;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry& e : cache)
      if (e.f == func && e.smem == smem && e.threads == threads && e.want == want) return e.got;
  }
  want = std::max(1, std::min(want, 16));
  int got = 0;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(want);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    int maxc = 0;
    if (cudaOccupancyMaxPotentialClusterSize(&maxc, func, &cfg) == cudaSuccess) {
      got = std::min(want, maxc);
      // the cluster size must divide the grid, which is one cluster
      while (got > 1 && (got & (got - 1))) --got;
    }
  }
  cudaGetLastError();  // a refused query leaves no sticky error
  std::lock_guard<std::mutex> lk(mu);
  cache.push_back({func, smem, threads, want, got});
  return got;
}

// `grid` CTAs running `func` in thread-block clusters of `cluster` CTAs.  The CTAs of a
// cluster are co-scheduled, so they may wait on each other; unlike cooperative launches,
// clusters issued from different streams run concurrently.
cudaError_t launch_cluster(const void* func, int cluster, int grid, int threads, size_t smem,
                           void** args, cudaStream_t s) {
  const int ctas = cluster;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, func, args);
}

template <typename T>
cudaError_t normalize_inplace(T* x, int64_t n, double* log_acc, int* status, double* scratch,
                              cudaStream_t s, int nb, bool shared_log) {
  cudaError_t err = cudaMemsetAsync(scratch, 0, sizeof(double) * nb, s);
  if (err != cudaSuccess) return err;
  const dim3 g(std::min(grid_for(n), std::max(1, 1024 / nb)), nb);
  note_launches(CBC_K_AUX, 2);
  sumsq_kernel<T><<<g, 256, 0, s>>>(x, n, scratch);
  scale_kernel<T><<<g, 256, 0, s>>>(x, n, scratch, log_acc, status, shared_log ? 1 : 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t scaled_adjoint(const T* V, int ldv, const double* lam, const int* k_dev, int n, T* L,
                           cudaStream_t s, int nb, int64_t l_bs) {
  note_launches(CBC_K_AUX, 1);
  scaled_adjoint_kernel<T><<<dim3(grid_for((int64_t)ldv * n), nb), 256, 0, s>>>(V, ldv, lam, k_dev,
                                                                              n, L, l_bs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t group_copy(T* const* ptrs, T* buf, int64_t stride, int64_t n, int nb, bool to_group,
                       cudaStream_t s) {
  note_launches(CBC_K_AUX, 1);
  group_copy_kernel<T><<<dim3(std::min(grid_for(n), std::max(1, 2048 / nb)), nb), 256, 0, s>>>(
      ptrs, buf, stride, n, to_group ? 1 : 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fill_identity(T* dst, int n, cudaStream_t s, int nb) {
  note_launches(CBC_K_AUX, 1);
  identity_kernel<T><<<dim3(grid_for((int64_t)n * n), nb), 256, 0, s>>>(dst, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t permute(const T* in, T* out, int rank, const int64_t* in_dims, const int* perm,
                    cudaStream_t s, int nb) {
  if (rank < 1 || rank > 8) return cudaErrorInvalidValue;
  int64_t in_stride[8];
  in_stride[rank - 1] = 1;
  for (int d = rank - 2; d >= 0; --d) in_stride[d] = in_stride[d + 1] * in_dims[d + 1];
  PermArgs a;
  a.rank = rank;
  int64_t total = 1;
  for (int d = 0; d < rank; ++d) {
    a.out_dims[d] = in_dims[perm[d]];
    a.in_stride_of_out[d] = in_stride[perm[d]];
    total *= a.out_dims[d];
  }
  if (total == 0) return cudaSuccess;
  note_launches(CBC_K_AUX, 1);
  permute_kernel<T><<<dim3(std::min(grid_for(total), std::max(1, 2048 / nb)), nb), 256, 0, s>>>(
      in, out, total, a);
  return cudaGetLastError();
}

cudaError_t widen_to_f64(const void* src, int src_dtype, void* dst, int64_t n_elem,
                         cudaStream_t s, int* nonfinite) {
  int64_t ns = n_elem * ((src_dtype == CBC_C64 || src_dtype == CBC_C128) ? 2 : 1);
  note_launches(CBC_K_AUX, 1);
  widen_kernel<<<grid_for(ns), 256, 0, s>>>(src, src_dtype, static_cast<double*>(dst), ns,
                                            nonfinite);
  return cudaGetLastError();
}

cudaError_t narrow_from_f64(const void* src, bool cplx, void* dst, int dst_dtype, int64_t n_elem,
                            cudaStream_t s) {
  int64_t ns = n_elem * (cplx ? 2 : 1);
  note_launches(CBC_K_AUX, 1);
  narrow_kernel<<<grid_for(ns), 256, 0, s>>>(static_cast<const double*>(src), dst, dst_dtype, ns);
  return cudaGetLastError();
}

template <typename T>
cudaError_t row_norms2(const T* W, int rows, int cols, int64_t ld, int64_t bs, double* out,
                       cudaStream_t s, int nb) {
  note_launches(CBC_K_AUX, 1);
  const int blocks = std::max(1, std::min(1024, (rows + 7) / 8));
  row_norms2_kernel<T><<<dim3(blocks, nb), 256, 0, s>>>(W, rows, cols, ld, bs, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t col_norms2(const T* W, int rows, int cols, int64_t ld, int64_t bs, double* out,
                       cudaStream_t s, int nb) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * (size_t)cols * nb, s);
  if (e != cudaSuccess) return e;
  note_launches(CBC_K_AUX, 1);
  const int chunks = std::max(1, std::min(std::max(1, 1024 / nb), (rows + 63) / 64));
  const int per = (rows + chunks - 1) / chunks;
  col_norms2_kernel<T><<<dim3(chunks, nb), dim3(32, 8), 0, s>>>(W, rows, cols, ld, bs, per, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t diff_sumsq(const T* A, int64_t a_bs, const T* B, T* C, int64_t n, double* out,
                       cudaStream_t s, int nb) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * nb, s);
  if (e != cudaSuccess) return e;
  note_launches(CBC_K_AUX, 1);
  diff_sumsq_kernel<T><<<dim3(std::min(grid_for(n), std::max(1, 1024 / nb)), nb), 256, 0, s>>>(
      A, a_bs, B, C, n, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t sum_squares(const T* x, int64_t n, double* out, cudaStream_t s, int nb) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * nb, s);
  if (e != cudaSuccess) return e;
  note_launches(CBC_K_AUX, 1);
  sumsq_kernel<T><<<dim3(std::min(grid_for(n), std::max(1, 1024 / nb)), nb), 256, 0, s>>>(x, n, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t scaled_adjoint_w(const T* V, int ldv, const double* w, int64_t w_bs, int k, int n,
                             T* L, int64_t l_bs, cudaStream_t s, int nb) {
  note_launches(CBC_K_AUX, 1);
  scaled_adjoint_w_kernel<T><<<dim3(grid_for((int64_t)k * n), nb), 256, 0, s>>>(V, ldv, w, w_bs,
                                                                               k, n, L, l_bs);
  return cudaGetLastError();
}

template <typename T>
cudaError_t scale_rows(T* X, int rows, int cols, int64_t bs, const double* norms2,
                       cudaStream_t s, int nb) {
  note_launches(CBC_K_AUX, 1);
  scale_rows_kernel<T><<<dim3(std::min(grid_for((int64_t)rows * cols), std::max(1, 2048 / nb)),
                              nb), 256, 0, s>>>(X, rows, cols, bs, norms2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t trace_real(const T* G, int g, int64_t bs, double* out, cudaStream_t s, int nb) {
  if (nb <= 0) return cudaSuccess;
  note_launches(CBC_K_AUX, 1);
  trace_kernel<T><<<nb, 256, 0, s>>>(G, g, bs, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t adjoint_copy(const T* in, int rows, int cols, T* out, cudaStream_t s) {
  if ((int64_t)rows * cols <= 0) return cudaSuccess;
  note_launches(CBC_K_AUX, 1);
  adjoint_kernel<T><<<grid_for((int64_t)rows * cols), 256, 0, s>>>(in, rows, cols, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t add_diagonal(T* G, int m, double shift, cudaStream_t s, int nb) {
  note_launches(CBC_K_AUX, 1);
  add_diag_kernel<T><<<dim3((m + 255) / 256, nb), 256, 0, s>>>(G, m, shift);
  return cudaGetLastError();
}

template <typename T>
cudaError_t copy_batched(const T* src, int64_t s_bs, T* dst, int64_t d_bs, int64_t n,
                         cudaStream_t s, int nb) {
  if (n <= 0) return cudaSuccess;
  note_launches(CBC_K_AUX, 1);
  copy_batched_kernel<T><<<dim3(std::min(grid_for(n), std::max(1, 2048 / nb)), nb), 256, 0, s>>>(
      src, s_bs, dst, d_bs, n);
  return cudaGetLastError();
}

// one thread per (j, col): the d products of the sketch row j with column col of Lp
template <typename T>
__global__ void sketch_kernel(const T* Lp, int c, int d, int64_t ncol, const T* om, int s,
                              int64_t lp_bs, int64_t om_bs, T* C, int64_t c_bs) {
  using O = ops<T>;
  const int b = blockIdx.z, j = blockIdx.y;
  Lp += (int64_t)b * lp_bs;
  om += (int64_t)b * om_bs;
  C += (int64_t)b * c_bs;
  const int cj = (c == 1) ? 0 : j;
  for (int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; col < ncol;
       col += (int64_t)gridDim.x * blockDim.x) {
    T acc = O::zero();
    for (int p = 0; p < d; ++p)
      acc = O::fma(Lp[((int64_t)cj * d + p) * ncol + col], om[(int64_t)p * s + j], acc);
    C[(int64_t)j * ncol + col] = acc;
  }
}

template <typename T>
cudaError_t sketch_contract(const T* Lp, int c, int d, int64_t ncol, const T* om, int s,
                            int64_t lp_bs, int64_t om_bs, T* C, int64_t c_bs, cudaStream_t st,
                            int nb) {
  if (s <= 0 || ncol <= 0 || nb <= 0) return cudaSuccess;
  if (c != 1 && c != s) return cudaErrorInvalidValue;
  note_launches(CBC_K_AUX, 1);
  const int gx = (int)std::min<int64_t>((ncol + 255) / 256, 1024);
  sketch_kernel<T><<<dim3(gx, s, nb), 256, 0, st>>>(Lp, c, d, ncol, om, s, lp_bs, om_bs, C, c_bs);
  return cudaGetLastError();
}

#define CBC_MISC_INST(T)                                                                     \
  template cudaError_t row_norms2<T>(const T*, int, int, int64_t, int64_t, double*,          \
                                     cudaStream_t, int);                                     \
  template cudaError_t col_norms2<T>(const T*, int, int, int64_t, int64_t, double*,          \
                                     cudaStream_t, int);                                     \
  template cudaError_t diff_sumsq<T>(const T*, int64_t, const T*, T*, int64_t, double*,      \
                                     cudaStream_t, int);                                     \
  template cudaError_t sum_squares<T>(const T*, int64_t, double*, cudaStream_t, int);        \
  template cudaError_t scaled_adjoint_w<T>(const T*, int, const double*, int64_t, int, int,  \
                                           T*, int64_t, cudaStream_t, int);                  \
  template cudaError_t copy_batched<T>(const T*, int64_t, T*, int64_t, int64_t, cudaStream_t, \
                                       int);                                                 \
  template cudaError_t scale_rows<T>(T*, int, int, int64_t, const double*, cudaStream_t, int); \
  template cudaError_t add_diagonal<T>(T*, int, double, cudaStream_t, int);                 \
  template cudaError_t adjoint_copy<T>(const T*, int, int, T*, cudaStream_t);               \
  template cudaError_t trace_real<T>(const T*, int, int64_t, double*, cudaStream_t, int);   \
  template cudaError_t sketch_contract<T>(const T*, int, int, int64_t, const T*, int, int64_t, \
                                          int64_t, T*, int64_t, cudaStream_t, int);
CBC_MISC_INST(double)
CBC_MISC_INST(zdbl)
#undef CBC_MISC_INST

template cudaError_t normalize_inplace<double>(double*, int64_t, double*, int*, double*,
                                               cudaStream_t, int, bool);
template cudaError_t normalize_inplace<zdbl>(zdbl*, int64_t, double*, int*, double*, cudaStream_t,
                                             int, bool);
template cudaError_t scaled_adjoint<double>(const double*, int, const double*, const int*, int,
                                            double*, cudaStream_t, int, int64_t);
template cudaError_t scaled_adjoint<zdbl>(const zdbl*, int, const double*, const int*, int, zdbl*,
                                          cudaStream_t, int, int64_t);
template cudaError_t permute<double>(const double*, double*, int, const int64_t*, const int*,
                                     cudaStream_t, int);
template cudaError_t permute<zdbl>(const zdbl*, zdbl*, int, const int64_t*, const int*,
                                   cudaStream_t, int);
template cudaError_t group_copy<double>(double* const*, double*, int64_t, int64_t, int, bool,
                                        cudaStream_t);
template cudaError_t group_copy<zdbl>(zdbl* const*, zdbl*, int64_t, int64_t, int, bool,
                                      cudaStream_t);
template cudaError_t fill_identity<double>(double*, int, cudaStream_t, int);
template cudaError_t fill_identity<zdbl>(zdbl*, int, cudaStream_t, int);

}  // namespace cbc
