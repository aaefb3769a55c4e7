// Householder reduction of the truncation Gram matrices to real symmetric tridiagonal
// form (the first stage of the eigensolver behind the compression of Sec. III A), one
// thread-block cluster per matrix.
//
// Layout: the P CTAs of a cluster own the rows r = rank + P t of the matrix and keep only
// their lower triangle (columns 0 .. r) in shared memory, packed row after row; with P = 4
// a 256 x 256 complex matrix in double-float pairs takes ~133 KB per CTA, so a batch of 32
// Gram matrices occupies 128 SMs in a single wave.
//
// Column j (H_j = I - tau v v^H, H^H x = beta e_1, beta real; x = A[j+1:, j]):
//   1. every CTA reads column j from the rows' owners through distributed shared memory
//      and computes v, tau, beta itself (the same data in the same order, so identical
//      values in every CTA: no broadcast needed);
//   2. every CTA forms its share of p = tau A v from its stored rows: each stored entry
//      A[r][c] (c <= r) contributes A[r][c] v_c to p_r and, below the diagonal,
//      conj(A[r][c]) v_r to p_c;
//   3. cluster barrier; every CTA adds the P shares in one fixed order (distributed
//      shared memory reads), forms w = p - (conj(tau)/2)(v^H p) v, and applies the rank-2
//      update A -= v w^H + w v^H to its own rows;
//   4. cluster barrier (column j+1 is final everywhere).
// Two hardware cluster barriers per column, no polling of global memory.  DF (the mixed
// path): the rows and every per-element quantity as double-float pairs, so all O(m) and
// O(m^2) work per column and every reduction runs in FP32 arithmetic with error-free
// transformations; FP64 only for the handful of Householder scalars, computed by one
// thread.  Otherwise FP64 throughout.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "df.cuh"
#include "kernels.cuh"
#include "planner.h"

namespace cg = cooperative_groups;

namespace cbc {
namespace {

constexpr int TCL_THREADS = 256;
constexpr int TCL_WARPS = TCL_THREADS / 32;
constexpr int TCL_CHUNK = 256;  // columns per pass of a warp (8 per lane)

template <typename T>
struct TriClArgs {
  const T* A;      // nb matrices m x m (row-major, Hermitian; lower triangle read)
  int m;
  double* d;       // per-matrix outputs, workspaces wb bytes apart:
  double* e;       //   diagonal, off-diagonal (beta_j), tau_j, and the reflectors
  T* tau;          //   V (row j: [j] = tau_j, [j+1] = 1, [c] = v_c)
  T* V;
  int64_t a_bs;    // elements between consecutive matrices A
  size_t wb;       // bytes between consecutive workspaces
  int rows_cap;    // stored elements of the largest share of rows
  int nr_cap;      // rows of the largest share
};

template <typename P>
__device__ __forceinline__ P* shift_bytes(P* p, size_t bytes) {
  return reinterpret_cast<P*>(reinterpret_cast<char*>(p) + bytes);
}

// Element type of the stored rows and of every per-element quantity (v, w, p and its
// shares), and the arithmetic on them: FP64 (T itself), or double-float pairs on the
// mixed path, where every per-element operation and every reduction runs on the FP32
// pipes and FP64 is left to the few scalars of each Householder step.
template <typename T, bool DF>
struct RowArith;
template <typename T>
struct RowArith<T, false> {
  using O = ops<T>;
  using E = T;
  using R = double;  // real quantities (norms)
  __device__ static __forceinline__ E cvt(T x) { return x; }
  __device__ static __forceinline__ T back(E x) { return x; }
  __device__ static __forceinline__ E mac(E a, E b, E c) { return O::fma(a, b, c); }
  __device__ static __forceinline__ E cj(E a) { return O::conj(a); }
  __device__ static __forceinline__ E zero() { return O::zero(); }
  __device__ static __forceinline__ E one() { return O::one(); }
  __device__ static __forceinline__ E add(E a, E b) { return a + b; }
  __device__ static __forceinline__ E mul(E a, E b) { return a * b; }
  __device__ static __forceinline__ E neg(E a) { return O::scale(-1.0, a); }
  __device__ static __forceinline__ E shfl(E a, int o) { return shfl_xor(a, o); }
  __device__ static __forceinline__ R rzero() { return 0.0; }
  __device__ static __forceinline__ R radd(R a, R b) { return a + b; }
  __device__ static __forceinline__ R abs2(E a) { return O::abs2(a); }
  __device__ static __forceinline__ double rback(R a) { return a; }
  __device__ static __forceinline__ R rshfl(R a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
};
template <typename T>
struct RowArith<T, true> {
  using O = ops<T>;
  using E = typename dfof<T>::type;
  using R = df1;
  __device__ static __forceinline__ E cvt(T x) { return to_df(x); }
  __device__ static __forceinline__ T back(E x) { return from_df(x); }
  __device__ static __forceinline__ E mac(E a, E b, E c) { return dff(a, b, c); }
  __device__ static __forceinline__ E cj(E a) { return dfconj(a); }
  __device__ static __forceinline__ E zero() { return E{}; }
  __device__ static __forceinline__ E one() {
    E x{};
    if constexpr (O::cplx) x.re.h = 1.f; else x.h = 1.f;
    return x;
  }
  __device__ static __forceinline__ E add(E a, E b) { return df_add(a, b); }
  __device__ static __forceinline__ E mul(E a, E b) { return dff(a, b, E{}); }
  __device__ static __forceinline__ E neg(E a) { return df_neg(a); }
  __device__ static __forceinline__ E shfl(E a, int o) { return df_shfl_xor(a, o); }
  __device__ static __forceinline__ R rzero() { return R{}; }
  __device__ static __forceinline__ R radd(R a, R b) { return df_add(a, b); }
  __device__ static __forceinline__ R abs2(E a) { return df_abs2(a); }
  __device__ static __forceinline__ double rback(R a) { return from_df(a); }
  __device__ static __forceinline__ R rshfl(R a, int o) { return df_shfl_xor(a, o); }
};

// offset of own row t (r = q + P t) in rank q's packed triangle: sum_{u<t} (q + P u + 1)
__device__ __forceinline__ int row_off(int q, int P, int t) {
  return t * (q + 1) + P * (t * (t - 1) / 2);
}

// Deterministic block sums: a butterfly per warp (lane 0's result is used), then the
// warps' results added in order by every thread: the same sequence of operations, hence
// the same value, in every CTA of the cluster.
template <typename AR>
__device__ __forceinline__ typename AR::E block_sum_e(typename AR::E x, typename AR::E* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = AR::add(x, AR::shfl(x, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = x;
  __syncthreads();
  typename AR::E s = red[0];
  for (int q = 1; q < TCL_WARPS; ++q) s = AR::add(s, red[q]);
  __syncthreads();
  return s;
}
template <typename AR>
__device__ __forceinline__ typename AR::R block_sum_r(typename AR::R x, typename AR::R* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = AR::radd(x, AR::rshfl(x, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = x;
  __syncthreads();
  typename AR::R s = red[0];
  for (int q = 1; q < TCL_WARPS; ++q) s = AR::radd(s, red[q]);
  __syncthreads();
  return s;
}

template <typename T, bool DF>
__global__ void __launch_bounds__(TCL_THREADS) tridiag_cluster_kernel(TriClArgs<T> a0) {
  using O = ops<T>;
  using AR = RowArith<T, DF>;
  using E = typename AR::E;
  using R = typename AR::R;
  cg::cluster_group cluster = cg::this_cluster();
  const int P = (int)cluster.num_blocks();
  const int cta = (int)cluster.block_rank();
  const int inst = blockIdx.x / P;
  const int m = a0.m;
  const T* A = a0.A + (int64_t)inst * a0.a_bs;
  const size_t off = (size_t)inst * a0.wb;
  double* d = shift_bytes(a0.d, off);
  double* e = shift_bytes(a0.e, off);
  T* tau_out = shift_bytes(a0.tau, off);
  T* V = shift_bytes(a0.V, off);

  extern __shared__ __align__(16) unsigned char smem_raw[];
  E* rows = reinterpret_cast<E*>(smem_raw);
  E* xE = rows + a0.rows_cap;            // column j
  E* vE = xE + m;                        // v
  E* ppE = vE + m;                       // this CTA's share of A v (read by the others)
  E* pE = ppE + m;                       // p = tau A v
  E* wE = pE + m;                        // w
  E* rpE = wE + m;                       // row sums of own rows
  E* wpartE = rpE + a0.nr_cap;           // [warp][m] column sums
  __shared__ E redE[TCL_WARPS];
  __shared__ R redR[TCL_WARPS];
  __shared__ T s_tau;
  __shared__ E s_tauE, s_scaleE, s_coefE;
  __shared__ int s_trivial;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nr = (m - cta + P - 1) / P;  // own rows r = cta + P t, t < nr
  for (int t = 0; t < nr; ++t) {
    const int r = cta + P * t;
    const T* src = A + (int64_t)r * m;
    E* dst = rows + row_off(cta, P, t);
    for (int c = tid; c <= r; c += TCL_THREADS) dst[c] = AR::cvt(src[c]);
  }
  cluster.sync();

  for (int j = 0; j < m - 1; ++j) {
    if (j % P == cta && tid == 0) d[j] = O::real(AR::back(rows[row_off(cta, P, j / P) + j]));
    // 1. column j below the diagonal, from its rows' owners
    for (int r = j + 1 + tid; r < m; r += TCL_THREADS) {
      const int q = r % P, t = r / P;
      xE[r] = cluster.map_shared_rank(rows, q)[row_off(q, P, t) + j];
    }
    __syncthreads();
    R part = AR::rzero();
    for (int c = j + 2 + tid; c < m; c += TCL_THREADS) part = AR::radd(part, AR::abs2(xE[c]));
    const R xn2e = block_sum_r<AR>(part, redR);
    if (tid == 0) {  // the Householder scalars, FP64, one thread
      const double xn2 = AR::rback(xn2e);
      const T alpha = AR::back(xE[j + 1]);
      const double ar = O::real(alpha), ai = O::imag(alpha);
      T tau, scale;
      double beta;
      const bool trivial = (xn2 == 0.0 && ai == 0.0);
      if (trivial) {
        tau = O::zero();
        beta = ar;
        scale = O::zero();
      } else {
        const double n2 = ar * ar + ai * ai + xn2;
        const double rn = rsqrt64(n2);  // 1 / ||x||
        const double nrm = n2 * rn;
        beta = (ar >= 0.0) ? -nrm : nrm;
        const double ib = (ar >= 0.0) ? -rn : rn;  // 1 / beta
        tau = O::make((beta - ar) * ib, -ai * ib);
        const double zr = ar - beta, zi = ai;
        const double iden = rcp64(zr * zr + zi * zi);
        scale = O::make(zr * iden, -zi * iden);  // 1 / (alpha - beta)
      }
      s_tau = tau;
      s_tauE = AR::cvt(tau);
      s_scaleE = AR::cvt(scale);
      s_trivial = trivial ? 1 : 0;
      if (cta == 0) {
        V[(int64_t)j * m + j] = tau;
        tau_out[j] = tau;
        e[j] = beta;
      }
    }
    const int t0 = (j + 1 > cta) ? (j + 1 - cta + P - 1) / P : 0;  // first own row beyond j
    for (int t = t0 + tid; t < nr; t += TCL_THREADS) rpE[t] = AR::zero();
    __syncthreads();
    {
      T* vrow = V + (int64_t)j * m;
      const E sc = s_scaleE;
      const bool triv = s_trivial != 0;
      for (int c = j + 1 + tid; c < m; c += TCL_THREADS) {
        const E v = (c == j + 1) ? AR::one() : (triv ? AR::zero() : AR::mul(xE[c], sc));
        vE[c] = v;
        if (c % P == cta) vrow[c] = AR::back(v);  // the reflectors, written by the rows' owners
      }
    }
    __syncthreads();

    // 2. this CTA's share of A v: warps over own rows, lanes over columns
    for (int base = j + 1; base < m; base += TCL_CHUNK) {
      E acc[TCL_CHUNK / 32];
#pragma unroll
      for (int q = 0; q < TCL_CHUNK / 32; ++q) acc[q] = AR::zero();
      for (int t = t0 + warp; t < nr; t += TCL_WARPS) {
        const int r = cta + P * t;
        if (r < base) continue;
        const E* row = rows + row_off(cta, P, t);
        const E vr = vE[r];
        E racc = AR::zero();
#pragma unroll
        for (int q = 0; q < TCL_CHUNK / 32; ++q) {
          const int c = base + lane + 32 * q;
          if (c <= r) {
            const E x = row[c];
            racc = AR::mac(x, vE[c], racc);                      // A[r][c] v_c       -> p_r
            if (c < r) acc[q] = AR::mac(AR::cj(x), vr, acc[q]);  // conj(A[r][c]) v_r -> p_c
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) racc = AR::add(racc, AR::shfl(racc, o));
        if (lane == 0) rpE[t] = AR::add(rpE[t], racc);
      }
#pragma unroll
      for (int q = 0; q < TCL_CHUNK / 32; ++q) {
        const int c = base + lane + 32 * q;
        if (c < m) wpartE[(size_t)warp * m + c] = acc[q];
      }
    }
    __syncthreads();
    for (int c = j + 1 + tid; c < m; c += TCL_THREADS) {
      E sum = (c % P == cta) ? rpE[c / P] : AR::zero();
      for (int w = 0; w < TCL_WARPS; ++w) sum = AR::add(sum, wpartE[(size_t)w * m + c]);
      ppE[c] = sum;
    }
    cluster.sync();  // every share of A v is ready

    // 3. p = tau A v from the P shares in a fixed order; v^H p; w; the rank-2 update
    E dp = AR::zero();
    {
      const E tauE = s_tauE;
      for (int c = j + 1 + tid; c < m; c += TCL_THREADS) {
        E sum = AR::zero();
        for (int q = 0; q < P; ++q) sum = AR::add(sum, cluster.map_shared_rank(ppE, q)[c]);
        const E p = AR::mul(tauE, sum);
        pE[c] = p;
        dp = AR::mac(AR::cj(vE[c]), p, dp);
      }
    }
    const E dot = block_sum_e<AR>(dp, redE);
    if (tid == 0) s_coefE = AR::cvt(O::scale(-0.5, O::conj(s_tau) * AR::back(dot)));
    __syncthreads();
    {
      const E coef = s_coefE;
      for (int c = j + 1 + tid; c < m; c += TCL_THREADS) wE[c] = AR::mac(coef, vE[c], pE[c]);
    }
    __syncthreads();
    for (int t = t0 + warp; t < nr; t += TCL_WARPS) {
      const int r = cta + P * t;
      E* row = rows + row_off(cta, P, t);
      const E nv = AR::neg(vE[r]);
      const E nw = AR::neg(wE[r]);
      for (int c = j + 1 + lane; c <= r; c += 32)
        row[c] = AR::mac(nw, AR::cj(vE[c]), AR::mac(nv, AR::cj(wE[c]), row[c]));
    }
    cluster.sync();  // column j + 1 is final in every CTA; the shares may be rewritten
  }
  if ((m - 1) % P == cta && tid == 0)
    d[m - 1] = O::real(AR::back(rows[row_off(cta, P, (m - 1) / P) + (m - 1)]));
}

template <typename T>
void cluster_shape(int m, int P, int* rows_cap, int* nr_cap) {
  int rc = 0, nc = 0;
  for (int q = 0; q < P; ++q) {
    const int nr = (m - q + P - 1) / P;
    const int cnt = nr * (q + 1) + P * (nr * (nr - 1) / 2);
    rc = std::max(rc, cnt);
    nc = std::max(nc, nr);
  }
  *rows_cap = rc;
  *nr_cap = nc;
}

template <typename T>
size_t cluster_smem(int m, int P, bool df) {
  int rc, nc;
  cluster_shape<T>(m, P, &rc, &nc);
  const size_t es = sizeof(T);  // a double-float element has the size of its FP64 one
  (void)df;
  return ((size_t)rc + (size_t)5 * m + nc + (size_t)TCL_WARPS * m) * es;
}

template <typename T>
const void* cluster_kernel(bool df) {
  return df ? (const void*)tridiag_cluster_kernel<T, true>
            : (const void*)tridiag_cluster_kernel<T, false>;
}

}  // namespace

template <typename T>
int tridiag_cluster_size(int m, bool df) {
  static_assert(sizeof(typename dfof<T>::type) == sizeof(T), "double-float element size");
  const void* k = cluster_kernel<T>(df);
  if (allow_max_smem(k) != cudaSuccess) return 0;
  for (int P : {4, 8, 16}) {
    const size_t smem = cluster_smem<T>(m, P, df);
    if (smem > 220 * 1024) continue;
    if (cluster_ctas(k, P, TCL_THREADS, smem) == P) return P;
  }
  return 0;
}

template <typename T>
cudaError_t tridiag_cluster(const T* A, int m, double* d, double* e, T* tau, T* V, int64_t a_bs,
                            size_t wb, int nb, int P, bool df, cudaStream_t s) {
  TriClArgs<T> a{A, m, d, e, tau, V, a_bs, wb, 0, 0};
  cluster_shape<T>(m, P, &a.rows_cap, &a.nr_cap);
  const void* k = cluster_kernel<T>(df);
  void* args[] = {&a};
  return launch_cluster(k, P, nb * P, TCL_THREADS, cluster_smem<T>(m, P, df), args, s);
}

template int tridiag_cluster_size<double>(int, bool);
template int tridiag_cluster_size<zdbl>(int, bool);
template cudaError_t tridiag_cluster<double>(const double*, int, double*, double*, double*,
                                             double*, int64_t, size_t, int, int, bool,
                                             cudaStream_t);
template cudaError_t tridiag_cluster<zdbl>(const zdbl*, int, double*, double*, zdbl*, zdbl*,
                                           int64_t, size_t, int, int, bool, cudaStream_t);

}  // namespace cbc
